"""Differentiable solve with a lifted initial datum (Sec. 3.1) on the GPU.

Workload square2d_p3_n48_b16: d = 2, p = 3, 48 elements (120,050 unknowns per right-hand side),
16 right-hand sides per launch, loss 0.5 ||u - u_target||^2.  Gradients of
the hand-written backward (adjoint solve + lifting transpose) are checked
against central finite differences of the GPU forward solve (h = 1e-6, 20
seeded directions, relative 1e-6) and against the oracle's gradient (direct
solves at a reduced mesh, the oracle PCG at full size; relative 1e-8).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.system import STProblem
from oracle.lifting import loss_and_grad, lift_matrix
from oracle.fd import FD
from oracle.solve import pcg
from paper_1809_10026_gb300 import synth

pytestmark = pytest.mark.gpu

PI = np.pi


def _inputs(prob, B, tag):
    """Seeded load vectors (sums of 8 separable sine modes of f), c0 and u_target."""
    Fs = []
    for b in range(B):
        a, k = synth.smooth_modes(1000 * tag + b, count=8, dims=prob.d + 1)
        terms = []
        for m in range(8):
            hs = [lambda x, kk=k[m, j]: np.sin(kk * PI * x) for j in range(prob.d)]
            terms.append((a[m], lambda t, kk=k[m, prob.d]: np.sin(kk * PI * t / 2), hs))
        Fs.append(prob.load_separable(terms))
    F = np.stack(Fs)
    c0 = np.stack([synth.grid_field(prob.n_s, 2000 * tag + b) for b in range(B)])
    ut = np.stack([synth.grid_field(prob.n_s + [prob.n_t], 3000 * tag + b, time_last=True) for b in range(B)])
    return F, c0, ut


def _grad_gpu(S, F, c0, ut, tol):
    from paper_1809_10026_gb300 import SolveFn
    Fg = torch.from_numpy(F.reshape(S.batch, -1)).cuda().requires_grad_(True)
    cg = torch.from_numpy(c0.reshape(S.batch, -1)).cuda().requires_grad_(True)
    u = SolveFn.apply(Fg, cg, S, tol, 500)
    loss = 0.5 * ((u - torch.from_numpy(ut.reshape(S.batch, -1)).cuda()) ** 2).sum()
    loss.backward()
    return float(loss.detach()), Fg.grad.cpu().numpy(), cg.grad.cpu().numpy(), u.detach().cpu().numpy()


def test_gradient_matches_oracle_reduced_mesh():
    import paper_1809_10026_gb300 as stls
    prob = STProblem(2, 3, 10)
    B = 3
    F, c0, ut = _inputs(prob, B, 1)
    S = stls.Solver(2, 3, 10, batch=B)
    L, dF, dc0, u = _grad_gpu(S, F, c0, ut, 1e-13)
    A = prob.assemble_A_kron()
    for b in range(B):
        Lr, dFr, dc0r, ur = loss_and_grad(prob, A, F[b], c0[b], ut[b])
        np.testing.assert_allclose(u[b], ur, rtol=0, atol=1e-10 * np.abs(ur).max())
        assert np.linalg.norm(dF[b] - dFr) <= 1e-8 * np.linalg.norm(dFr)
        assert np.linalg.norm(dc0[b] - dc0r) <= 1e-8 * np.linalg.norm(dc0r)


def test_gradients_square2d_p3_n48_b16():
    import paper_1809_10026_gb300 as stls
    prob = STProblem(2, 3, 48)
    B = 16
    F, c0, ut = _inputs(prob, B, 5)
    S = stls.Solver(2, 3, 48, batch=B)
    assert S.N == 120050 and S.batch == 16
    L, dF, dc0, u = _grad_gpu(S, F, c0, ut, 1e-12)
    # central differences of the GPU forward solve along 20 seeded directions
    rng = synth.rng(55)
    for _ in range(20):
        vF = rng.standard_normal(F.shape)
        vc = rng.standard_normal(c0.shape)
        h = 1e-6
        Lp = _grad_gpu(S, F + h * vF, c0 + h * vc, ut, 1e-12)[0]
        Lm = _grad_gpu(S, F - h * vF, c0 - h * vc, ut, 1e-12)[0]
        fd = (Lp - Lm) / (2 * h)
        an = float(np.sum(dF * vF) + np.sum(dc0 * vc))
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-30), (fd, an)
    # oracle gradient for two right-hand sides: its own PCG with the FD preconditioner
    fdp = FD(prob)
    G = lift_matrix(prob)
    for b in (0, 11):
        w, _, _ = pcg(prob.apply_A_kron, fdp.apply, F[b] - G @ c0[b], 1e-13, 500)
        ur = w + np.kron(np.ones(prob.n_t), c0[b])
        g = ur - ut[b]
        lam, _, _ = pcg(prob.apply_A_kron, fdp.apply, g, 1e-13, 500)
        dc0r = g.reshape(prob.n_t, prob.N_s).sum(axis=0) - G.T @ lam
        assert np.linalg.norm(u[b] - ur) <= 1e-9 * np.linalg.norm(ur)
        assert np.linalg.norm(dF[b] - lam) <= 1e-8 * np.linalg.norm(lam)
        assert np.linalg.norm(dc0[b] - dc0r) <= 1e-8 * np.linalg.norm(dc0r)


@pytest.mark.parametrize("d,p,n_el,T", [(1, 2, 9, 1.0), (2, 3, 6, 0.7), (3, 2, 3, 1.4)])
def test_lift_calls_match_oracle(d, p, n_el, T):
    """stls_lifted_rhs = F - G c0 and stls_lift_add = w + 1_{n_t} x c0 (Sec. 3.1
    lifting), two right-hand sides, against the oracle's G; the addition is
    one rounding per entry, so it is compared exactly."""
    import paper_1809_10026_gb300 as stls
    prob = STProblem(d, p, n_el, T)
    B = 2
    S = stls.Solver(d, p, n_el, T, batch=B)
    rng = np.random.default_rng(7)
    F = rng.standard_normal((B, prob.N))
    c0 = rng.standard_normal((B, prob.N_s))
    w = rng.standard_normal((B, prob.N))
    G = lift_matrix(prob)
    absG = abs(G)
    rhs = S.lifted_rhs(torch.from_numpy(F).cuda(), torch.from_numpy(c0).cuda()).cpu().numpy()
    u = S.lift_add(torch.from_numpy(w).cuda(), torch.from_numpy(c0).cuda()).cpu().numpy()
    for b in range(B):
        ref = F[b] - G @ c0[b]
        bound = 1e-13 * (np.abs(F[b]) + absG @ np.abs(c0[b]))
        assert np.all(np.abs(rhs[b] - ref) <= bound)
        assert np.array_equal(u[b], w[b] + np.kron(np.ones(prob.n_t), c0[b]))
    # the output may not overlap an input
    from paper_1809_10026_gb300 import _lib
    Fg, cg = torch.from_numpy(F).cuda(), torch.from_numpy(c0).cuda()
    assert S.lib.stls_lifted_rhs(S.ctx, S._ptr(Fg), S._ptr(cg), S._ptr(Fg)) == _lib.STLS_EINVAL
    assert S.lib.stls_lift_add(S.ctx, S._ptr(Fg), S._ptr(cg), S._ptr(Fg)) == _lib.STLS_EINVAL
