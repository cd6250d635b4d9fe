"""GPU checks of the solver's reporting and host-side interfaces through the
C ABI: the host-buffer solve (the bench's end-to-end path) against the
device solve, the context's factor copies and launch counter, the residual
history against the oracle PCG's, and failure detection with an indefinite
preconditioner (a host-side override of the eigenvalues)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.system import STProblem
from oracle.fd import FD
from oracle.solve import direct_solve, pcg
from paper_1809_10026_gb300 import synth

pytestmark = pytest.mark.gpu


def _solver(*a, **k):
    import paper_1809_10026_gb300 as stls
    return stls.Solver(*a, **k)


def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("kw", [dict(), dict(precision="tf32", refine=True)], ids=["fp64", "tf32_refine"])
def test_solve_host_matches_device_solve(kw):
    """stls_solve_host (host F and u, copies inside the call; the bench's
    end-to-end path) gives bit for bit the device solve's u and iteration
    counts (same kernels, fixed-order reductions), with pageable numpy arrays
    and with pinned buffers, and the direct solve's u to the tolerance."""
    B = 2
    prob = STProblem(2, 3, 6)
    S = _solver(2, 3, 6, batch=B, **kw)
    F = synth.uniform(prob.N, 21, batch=B)
    u_dev, info_d = S.solve(_cuda(F), tol=1e-12, maxit=300)
    u_dev = u_dev.cpu().numpy()
    u_host, info_h = S.solve_host(F, tol=1e-12, maxit=300)
    assert np.array_equal(u_host.reshape(B, prob.N), u_dev)
    assert [i["iters"] for i in info_h] == [i["iters"] for i in info_d]
    Fh = torch.from_numpy(F).pin_memory()
    uh = torch.empty_like(Fh).pin_memory()
    info_p = S.solve_host_ptr(Fh.data_ptr(), uh.data_ptr(), tol=1e-12, maxit=300)
    assert np.array_equal(uh.numpy(), u_dev) and info_p[0]["status"] == "ok"
    A = prob.assemble_A_kron()
    for b in range(B):
        ref = direct_solve(A, F[b])
        assert np.linalg.norm(u_host.reshape(B, -1)[b] - ref) <= 1e-8 * np.linalg.norm(ref)


@pytest.mark.parametrize("tol", [1e-8, 1e-11])
def test_solve_host_refinement_copy_overlap(tol):
    """Refinement form: stls_solve_host copies u to the host while the FP64
    residual that may confirm convergence runs, and again if a later outer
    step changes u.  At 1e-11 several outer steps take an FP64 residual, so
    early copies are superseded; the host u must still equal the device
    solve's bit for bit, on repeated calls into the same buffer."""
    prob = STProblem(3, 3, 12)
    S = _solver(3, 3, 12, precision="tf32", refine=True)
    F = synth.uniform(prob.N, 23)
    u_dev, info_d = S.solve(_cuda(F), tol=tol, maxit=400)
    u_dev = u_dev.cpu().numpy()
    assert info_d[0]["status"] == "ok" and info_d[0]["outer"] >= (3 if tol < 1e-10 else 2)
    Fh = torch.from_numpy(F).pin_memory()
    uh = torch.full_like(Fh, float("nan")).pin_memory()
    for _ in range(2):
        info_h = S.solve_host_ptr(Fh.data_ptr(), uh.data_ptr(), tol=tol, maxit=400)
        assert info_h[0]["iters"] == info_d[0]["iters"] and info_h[0]["outer"] == info_d[0]["outer"]
        assert np.array_equal(uh.numpy(), u_dev)
        uh.fill_(float("nan"))


def test_context_factors_and_launch_count():
    """stls_get_factor returns the context's copies of the host setup's 1D
    factors (bitwise those of stls_host_factor), and the launch counter
    advances by the kernels one fused A x launches (slice, z and t passes)."""
    import paper_1809_10026_gb300 as stls
    S = _solver(3, 2, [4, 5, 3], 0.8)
    for which in ("mass", "stiff", "bilap", "eigvec", "eigval"):
        for k in range(3):
            ref = stls.host_factor(which, k, 3, 2, [4, 5, 3], T=0.8)
            assert np.array_equal(S.factor(which, k), ref)
    for which in ("mass", "stiff", "eigvec", "eigval", "end", "integral"):
        ref = stls.host_factor(which, 3, 3, 2, [4, 5, 3], T=0.8)
        assert np.array_equal(S.factor(which, 3), ref)
    x = _cuda(synth.uniform(S.N, 5))
    n0 = S.launch_count()
    S.apply_A(x)
    torch.cuda.synchronize()
    assert S.launch_count() - n0 == 3


def test_indefinite_preconditioner_reports_breakdown():
    """Failure detection on the host side: eigenvalues overridden so that one
    entry of the eigenvalue tensor is slightly negative make P indefinite;
    (z, r) < 0 then (the oracle's FD with the same values gives (z, r) < 0 for
    every seed tried), and the solve stops with a breakdown status instead of
    iterating on.  The context stays usable."""
    import paper_1809_10026_gb300 as stls
    prob = STProblem(2, 3, 4)
    S = _solver(2, 3, 4)
    F = synth.uniform(prob.N, 0)
    u, info = S.solve(_cuda(F), tol=1e-10)
    assert info[0]["status"] == "ok"
    l1, l2, lt = S.factor("eigval", 0), S.factor("eigval", 1), S.factor("eigval", 2)
    s = l1[0] + l2[0]
    bad = lt.copy()
    bad[0] = -s - 1e-6 * (s + abs(lt[0]))
    fd = FD(prob)
    fd.lam_t = bad.copy()
    assert F @ fd.apply(F) < 0
    S.override_eigenvalues(2, bad)
    assert np.array_equal(S.factor("eigval", 2), bad)
    u, info = S.solve(_cuda(F), tol=1e-10, check=False)
    assert info[0]["status"] == "breakdown"
    with pytest.raises(RuntimeError, match="breakdown"):
        S.solve(_cuda(F), tol=1e-10)
    S.override_eigenvalues(2, lt)  # restored: the context solves again
    u, info = S.solve(_cuda(F), tol=1e-10)
    assert info[0]["status"] == "ok"
    with pytest.raises(RuntimeError):
        stls.Solver(2, 3, 4, precision="bf16").override_eigenvalues(2, lt)


@pytest.mark.parametrize("d,p,n_el", [(1, 3, 12), (2, 2, 7), (3, 3, 4)])
def test_residual_history_matches_oracle_pcg(d, p, n_el):
    """The PCG residual recurrence step by step: the relative residual of every
    iteration (stls_residual_history) equals the oracle PCG's (same algorithm,
    FP64, same stopping rule).  The two differ by rounding and by their
    eigenvectors (~1e-12 relative here), far below the 1e-6 bound; a wrong
    term or index would change the sequence at O(1)."""
    prob = STProblem(d, p, n_el)
    F = synth.uniform(prob.N, 50 + d)
    S = _solver(d, p, n_el)
    assert len(S.residual_history()) == 0  # before any solve
    u, info = S.solve(_cuda(F), tol=1e-11, maxit=200)
    h = S.residual_history()
    _, it, h_ref = pcg(prob.apply_A_kron, FD(prob).apply, F, 1e-11, 200)
    assert info[0]["iters"] == it == len(h) - 1
    np.testing.assert_allclose(h, h_ref, rtol=1e-6, atol=0)
    assert h[-1] == info[0]["rel_res"] <= 1e-11


def test_residual_history_refinement_and_batch():
    """Refinement form: one entry per outer step, ending with the FP64 residual
    the solve reports; a zero right-hand side has the history [0]."""
    B = 2
    prob = STProblem(3, 3, 5)
    F = synth.uniform(prob.N, 61, batch=B)
    F[1] = 0.0
    S = _solver(3, 3, 5, precision="tf32", refine=True, batch=B)
    u, info = S.solve(_cuda(F), tol=1e-10, maxit=400)
    h0, h1 = S.residual_history(0), S.residual_history(1)
    assert len(h0) == info[0]["outer"] + 1 and h0[0] == 1.0
    assert h0[-1] == info[0]["rel_res"]
    assert h0[-1] <= 1e-10 and np.all(np.diff(h0) < 0)
    assert list(h1) == [0.0]


@pytest.mark.parametrize("form", [("tf32", 1), ("bf16", 2)], ids=["tf32", "bf16_batch2"])
def test_graph_inner_loop_matches_host_loop(form):
    """The refinement form runs each inner FP32 loop as one CUDA-graph launch
    (while node, condition set on the device) unless phase timing is on, when
    the host drives the loop step by step.  Both run the same kernels in the
    same order: u, the iteration counts and the residual history must agree
    bit for bit, and the launch counter must count the graph's kernels."""
    prec, B = form
    prob = STProblem(3, 3, 10)
    S = _solver(3, 3, 10, precision=prec, refine=True, batch=B)
    F = synth.uniform(prob.N, 31, batch=B).reshape(B, prob.N)
    if B > 1:
        # a smooth load converges in other steps than the random one, so one
        # right-hand side leaves the loop while the other goes on
        s = lambda x: np.sin(np.pi * x)
        F[1] = prob.load_separable([(1.0, np.cos, [s, s, s]), (3 * np.pi ** 2, np.sin, [s, s, s])])
    Fg = _cuda(F.reshape(-1) if B == 1 else F)
    l0 = S.launch_count()
    u_graph, info_g = S.solve(Fg, tol=1e-10, maxit=400)
    l_graph = S.launch_count() - l0
    hist_g = [S.residual_history(b) for b in range(B)]
    S.enable_timing(True)
    l0 = S.launch_count()
    u_host, info_h = S.solve(Fg, tol=1e-10, maxit=400)
    l_host = S.launch_count() - l0
    hist_h = [S.residual_history(b) for b in range(B)]
    S.enable_timing(False)
    assert torch.equal(u_graph, u_host)
    for b in range(B):
        assert info_g[b]["status"] == "ok" and info_h[b]["status"] == "ok"
        for k in ("iters", "outer", "outer_df"):
            assert info_g[b][k] == info_h[b][k]
        assert info_g[b]["true_rel_res"] == info_h[b]["true_rel_res"]
        assert np.array_equal(hist_g[b], hist_h[b])
    if B > 1:
        assert len(hist_g[0]) != len(hist_g[1]) or not np.array_equal(hist_g[0], hist_g[1])
    # the graph adds one condition kernel per inner step
    assert l_graph == l_host + info_g[0]["iters"]
