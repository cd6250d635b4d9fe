"""GPU check of the time-slab decomposition's local operations: P = 2 to 4
ranks held in one process exchange through LoopbackComm (a hand-over of
tensors: no kernel waits on another), each rank's arithmetic in the
library's slab calls; the distributed A x, P^{-1} r and PCG solve equal the
context's own operators and the oracle's."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.system import STProblem
from oracle.fd import FD
from oracle.solve import direct_solve
from paper_1809_10026_gb300 import synth
from paper_1809_10026_gb300.timeslab import Partition, LoopbackComm, TimeSlabPCG, GpuLocal

pytestmark = pytest.mark.gpu


def _split(x, part, B):
    X = x.reshape(B, part.n_t, part.N_s)
    return {r: X[:, t0:t1].contiguous() for r, (t0, t1) in enumerate(part.t)}


def _join(parts, part, B):
    return torch.cat([parts[r] for r in range(part.P)], dim=1).reshape(B, -1)


@pytest.mark.parametrize("P,d,p,n_el,T", [(2, 3, 3, 6, 1.0), (3, 2, 2, 6, 1.2), (4, 1, 2, 13, 1.0),
                                           (2, 2, 4, 8, 1.0)])
def test_gpu_timeslab_operators(P, d, p, n_el, T):
    import paper_1809_10026_gb300 as stls
    prob = STProblem(d, p, n_el, T)
    B = 2
    S = stls.Solver(d, p, n_el, T, batch=B)
    part = Partition(S.n_t, S.N_s, P, p)
    ts = TimeSlabPCG(part, {r: GpuLocal(S) for r in range(P)}, LoopbackComm())
    x = torch.from_numpy(synth.uniform(S.N, 61, batch=B).reshape(B, S.N)).cuda()
    y = _join(ts.apply_A(_split(x, part, B)), part, B)
    z = _join(ts.apply_precond(_split(x, part, B)), part, B)
    y0, z0 = S.apply_A(x), S.apply_precond(x)
    torch.cuda.synchronize()
    y, z, y0, z0 = (v.cpu().numpy() for v in (y, z, y0, z0))
    A, fd = prob.assemble_A_kron(), FD(prob)
    xs = x.cpu().numpy()
    for b in range(B):
        ref = A @ xs[b]
        assert np.abs(y[b] - ref).max() <= 1e-13 * np.abs(ref).max()
        assert np.abs(y[b] - y0[b]).max() <= 1e-13 * np.abs(ref).max()
        refz = fd.apply(xs[b])
        # the library's eigenvectors against LAPACK's: the FD parity bound of the cube
        assert np.abs(z[b] - z0[b]).max() <= 1e-13 * np.abs(z0[b]).max()
        assert np.abs(z[b] - refz).max() <= 1e-9 * np.abs(refz).max()


def test_gpu_timeslab_solve():
    import paper_1809_10026_gb300 as stls
    prob = STProblem(3, 2, 5)      # n_t = 6, p_t = 2: three slabs of two slices
    B = 2
    S = stls.Solver(3, 2, 5, batch=B)
    part = Partition(S.n_t, S.N_s, 3, 2)
    ts = TimeSlabPCG(part, {r: GpuLocal(S) for r in range(3)}, LoopbackComm())
    F = synth.uniform(S.N, 62, batch=B).reshape(B, S.N)
    u, it, rel = ts.solve(_split(torch.from_numpy(F).cuda(), part, B), 1e-12, 300)
    u = _join(u, part, B).cpu().numpy()
    A = prob.assemble_A_kron()
    _, info = S.solve(torch.from_numpy(F).cuda(), tol=1e-12, maxit=300)
    for b in range(B):
        ref = direct_solve(A, F[b])
        assert rel[b] <= 1e-12 and np.linalg.norm(u[b] - ref) <= 1e-10 * np.linalg.norm(ref)
    # the same PCG as the context's solve (sums in another order): the same iteration count within one
    assert abs(it - max(i["iters"] for i in info)) <= 1
