"""GPU runs on the benchmark's mesh (3D, 64 elements per direction, 17 to
20.5 million unknowns), checked by the oracle: Table 1's iteration counts of
P + CG at n_sub = 64, the benchmark's own solve (TF32 refinement form) with
its residual recomputed by the oracle, and the degree sweep at the
benchmark's size (p = 2..6, 67 - p elements, N = 18,125,250 for every p)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.system import STProblem
from paper_1809_10026_gb300 import synth

pytestmark = pytest.mark.gpu

PI = np.pi
TABLE1_N64 = 13  # Table 1, n_sub = 64: 13 iterations for p = 2, 3, 4, 5


def _solver(*a, **k):
    import paper_1809_10026_gb300 as stls
    return stls.Solver(*a, **k)


@pytest.mark.parametrize("p", [2, 3, 4, 5])
def test_table1_iterations_n_sub_64(p):
    """Table 1 at n_sub = 64 (u = sin sin sin sin(t), tol 1e-8, x0 = 0): 13
    iterations.  The oracle's PCG also takes 13 there, with the residual of
    iteration 12 at 1.30e-8 to 1.48e-8, so the count does not hinge on
    rounding."""
    prob = STProblem(3, p, 64)
    s = lambda x: np.sin(PI * x)
    F = prob.load_separable([(1.0, np.cos, [s, s, s]), (3 * PI ** 2, np.sin, [s, s, s])])
    S = _solver(3, p, 64)
    u, info = S.solve(torch.from_numpy(F).cuda(), tol=1e-8, maxit=100)
    assert info[0]["status"] == "ok" and info[0]["iters"] == TABLE1_N64


@pytest.mark.parametrize("fp64_residuals", [False, True])
def test_headline_solve_cube3d_p3_n64_tf32_refinement(fp64_residuals):
    """The bench's solve as the bench runs it: 3D, p = 3, 64 elements
    (18,125,250 unknowns), F ~ U[-1,1] (seed tag 4), TF32 refinement form,
    tol 1e-8.  The oracle recomputes the residual ||F - A u|| / ||F|| of the
    returned u with its own Kronecker-factored A: it is below the tolerance and
    agrees with the library's FP64 residual to 1e-11 (both FP64; their
    rounding differs by ~1e-14 relative to ||F|| at the solution)."""
    prob = STProblem(3, 3, 64)
    S = _solver(3, 3, 64, precision="tf32", refine=True, fp64_residuals=fp64_residuals)
    assert S.N == prob.N == 18125250
    F = synth.uniform(prob.N, 4)
    u, info = S.solve(torch.from_numpy(F).cuda(), tol=1e-8, maxit=200)
    it = info[0]
    assert it["status"] == "ok" and it["true_rel_res"] <= 1e-8
    assert it["iters"] <= 30 and it["outer"] <= 4
    assert (it["outer_df"] == 0) if fp64_residuals else (it["outer_df"] >= 1)
    u = u.cpu().numpy()
    res = np.linalg.norm(F - prob.apply_A_kron(u)) / np.linalg.norm(F)
    assert res <= 1e-8 + 1e-11 and abs(res - it["true_rel_res"]) <= 1e-11, (res, it)


@pytest.mark.parametrize("p", [2, 3, 4, 5, 6])
def test_degree_sweep_fixed_dofs(p):
    """Degree sweep at fixed N = 18,125,250 (p = 2..6, 67 - p elements per
    direction; F ~ U[-1,1], tol 1e-8): the headline form (TF32 refinement) and
    the FP64 PCG converge, and the oracle's own A recomputes each returned
    solution's residual.  Sec. 4.5: the FD cost does not depend on p, so the
    FP64 PCG's iteration count stays in the range of Table 1 (12-13 on the
    manufactured load; 17 here on the random one for p = 3)."""
    n_el = 67 - p
    prob = STProblem(3, p, n_el)
    assert prob.N == 18125250
    F = synth.uniform(prob.N, 4)
    nF = np.linalg.norm(F)
    Fg = torch.from_numpy(F).cuda()
    for kw, max_iters in ((dict(precision="tf32", refine=True), 40), (dict(), 25)):
        S = _solver(3, p, n_el, **kw)
        u, info = S.solve(Fg, tol=1e-8, maxit=400)
        it = info[0]
        assert it["status"] == "ok" and it["true_rel_res"] <= 1e-8 and it["iters"] <= max_iters, (kw, it)
        res = np.linalg.norm(F - prob.apply_A_kron(u.cpu().numpy())) / nF
        print("p=%d %s: iterations %d (outer %d), residual %.3e (oracle %.3e)"
              % (p, kw.get("precision", "fp64"), it["iters"], it["outer"], it["true_rel_res"], res))
        assert res <= 1e-8 + 1e-11 and abs(res - it["true_rel_res"]) <= 1e-11, (kw, res, it)
        del u, S
