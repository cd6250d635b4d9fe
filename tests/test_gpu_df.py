"""GPU parity of the double-float A x (FP32 pairs) and of the refinement form's
provisional outer residuals, through the C ABI.

The double-float product carries every value as h + l (two FP32 numbers,
about 48 significant bits).  Each banded dot product accumulates its exact
FP32 products by TwoSum with one FP32 low sum, so one stage errs by a few
2^-48 of the sum of its absolute terms; four stages (directions 1-3 and time)
chain them.  With B = (sum of the absolute Kronecker terms of the fused
product) |x|, the largest error measured on GB300 over the cases below is
about 2^-46 B_i; the test bound is 2^-42 B_i, 2^18 times below the error of
plain FP32 arithmetic (~2^-24 B_i) that a dropped low part or cross term
would give.
"""
import numpy as np
import pytest
import scipy.sparse as sp

torch = pytest.importorskip("torch")

from oracle.system import STProblem, kron_all
from paper_1809_10026_gb300 import synth

pytestmark = pytest.mark.gpu

BOUND = 2.0 ** -42


def _solver(*a, **k):
    import paper_1809_10026_gb300 as stls
    return stls.Solver(*a, **k)


def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def abs_terms(prob):
    """Sum of |Kronecker term| over the terms the fused product evaluates:
    |K_t| x |M_s| + |M_t| x (sum_k |J_k| + 2 sum_{k<l} |K_k| |K_l|) + |W_t| x sum_k |K_k|
    (M in the other directions)."""
    tm, sd, d = prob.time, prob.space, prob.d
    ab = lambda W: sp.csr_matrix(np.abs(W))
    absM = [ab(s.M) for s in sd]
    J = 0
    L = 0
    for k in range(d):
        mats = list(absM)
        mats[k] = ab(sd[k].J)
        J = J + kron_all(mats)
        mats = list(absM)
        mats[k] = ab(sd[k].K)
        L = L + kron_all(mats)
        for l in range(k + 1, d):
            mats = list(absM)
            mats[k] = ab(sd[k].K)
            mats[l] = ab(sd[l].K)
            J = J + 2 * kron_all(mats)
    return sp.csr_matrix(sp.kron(ab(tm.K), kron_all(absM)) + sp.kron(ab(tm.M), J) + sp.kron(ab(tm.W), L))


CASES = [dict(d=2, p=2, n_el=7), dict(d=2, p=3, n_el=9, T=1.3), dict(d=2, p=5, n_el=4),
         dict(d=3, p=2, n_el=4), dict(d=3, p=3, n_el=5, T=0.9), dict(d=3, p=4, n_el=3),
         dict(d=2, p=2, n_el=1), dict(d=3, p=5, n_el=1),
         dict(d=3, p=3, n_el=[4, 3, 5], T=1.1, p_t=1, n_el_t=7),
         dict(d=2, p=2, n_el=[6, 9], T=0.5, p_t=5, n_el_t=3),
         dict(d=2, p=3, n_el=[40, 7]),
         dict(d=3, p=6, n_el=2), dict(d=2, p=6, n_el=[5, 3], T=0.8, p_t=6, n_el_t=2),
         dict(d=2, p=2, n_el=4, p_t=6, n_el_t=3)]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "-".join(f"{k}{v}" for k, v in c.items()))
def test_apply_A_df_matches_oracle(case):
    kw = {k: case[k] for k in ("T", "p_t", "n_el_t") if k in case}
    prob = STProblem(case["d"], case["p"], case["n_el"], **kw)
    S = _solver(case["d"], case["p"], case["n_el"], precision="bf16", refine=True, batch=2, **kw)
    x = synth.uniform(prob.N, 41, batch=2).reshape(2, prob.N)
    x[1] *= 3.0e5  # a second magnitude: the FP32 parts scale with it
    y = S.apply_A_df(_cuda(x)).cpu().numpy().reshape(2, prob.N)
    A = prob.assemble_A_kron()
    Babs = abs_terms(prob)
    worst = 0.0
    for b in range(2):
        ref = A @ x[b]
        B = Babs @ np.abs(x[b])
        err = np.abs(y[b] - ref)
        worst = max(worst, float(np.max(err / B)))
        assert np.all(err <= BOUND * B), float(np.max(err / B))
    print("max |y - Ax| / B:", worst, "= 2^%.1f" % np.log2(max(worst, 1e-300)))


def test_apply_A_df_needs_refinement_context():
    S = _solver(3, 2, 3)  # FP64 form: no double-float operator
    x = _cuda(synth.uniform(S.N, 1))
    with pytest.raises(RuntimeError, match="apply_A_df"):
        S.apply_A_df(x)
    S1 = _solver(1, 2, 5, precision="bf16", refine=True)  # one spatial direction: no fused A x
    with pytest.raises(RuntimeError, match="apply_A_df"):
        S1.apply_A_df(_cuda(synth.uniform(S1.N, 1)))


def test_apply_A_df_zero_and_exact_values():
    """x = 0 gives y = 0 exactly; x with few significant bits (exact in the
    high parts) on the smallest degree and mesh."""
    prob = STProblem(2, 2, 1)
    S = _solver(2, 2, 1, precision="bf16", refine=True)
    z = S.apply_A_df(_cuda(np.zeros(prob.N))).cpu().numpy()
    assert np.array_equal(z, np.zeros(prob.N))
    x = np.round(synth.uniform(prob.N, 5) * 64) / 64
    ref = prob.assemble_A_kron() @ x
    y = S.apply_A_df(_cuda(x)).cpu().numpy()
    B = abs_terms(prob) @ np.abs(x)
    assert np.all(np.abs(y - ref) <= BOUND * B)


def test_df_residual_accuracy_cube3d_p3_n64():
    """3D, p = 3, 64 elements (18,125,250 DoF).  (1) Random x: the double-float
    product agrees with the FP64 one normwise to 1e-12.  (2) The solution of a
    refinement solve: F - A_df u differs from the FP64 residual F - A u by
    less than 1e-10 ||F||, 100 times below the 1e-8 floor under which the solver
    stops taking provisional residuals."""
    S = _solver(3, 3, 64, precision="bf16", refine=True)
    x = _cuda(synth.uniform(S.N, 9))
    y64 = S.apply_A(x)
    ydf = S.apply_A_df(x)
    rel = (torch.linalg.norm(ydf - y64) / torch.linalg.norm(y64)).item()
    assert rel <= 1e-12, rel
    F = _cuda(synth.uniform(S.N, 4))
    u, info = S.solve(F, tol=1e-8, maxit=200)
    assert info[0]["status"] == "ok" and info[0]["true_rel_res"] <= 1e-8
    assert info[0]["outer_df"] >= 1
    r64 = F - S.apply_A(u)
    rdf = F - S.apply_A_df(u)
    nF = torch.linalg.norm(F).item()
    delta = torch.linalg.norm(rdf - r64).item() / nF
    print("random x: rel diff", rel, "| residual of the solution: ||r_df - r_64|| / ||F|| =", delta,
          "| ||r_64|| / ||F|| =", torch.linalg.norm(r64).item() / nF, "| outer", info[0]["outer"],
          "of which double-float", info[0]["outer_df"])
    assert delta <= 1e-10, delta


@pytest.mark.parametrize("form", ["bf16", "tf32"])
def test_refinement_fp64_residuals_option(form):
    """fp64_residuals = 1: every outer residual in FP64 (no provisional double-float
    ones); the solve reaches the same tolerance and agrees with the default."""
    pi = np.pi
    prob = STProblem(3, 4, 32)
    s = lambda x: np.sin(pi * x)
    F = _cuda(prob.load_separable([(1.0, np.cos, [s, s, s]), (3 * pi ** 2, np.sin, [s, s, s])]))
    S64 = _solver(3, 4, 32, precision=form, refine=True, fp64_residuals=True)
    u64, i64 = S64.solve(F, tol=1e-12, maxit=800)
    assert i64[0]["status"] == "ok" and i64[0]["true_rel_res"] <= 1e-12 and i64[0]["outer_df"] == 0
    Sdf = _solver(3, 4, 32, precision=form, refine=True)
    udf, idf = Sdf.solve(F, tol=1e-12, maxit=800)
    assert idf[0]["status"] == "ok" and idf[0]["true_rel_res"] <= 1e-12 and idf[0]["outer_df"] >= 1
    rel = (torch.linalg.norm(udf - u64) / torch.linalg.norm(u64)).item()
    assert rel <= 1e-8, rel
    with pytest.raises(RuntimeError, match="apply_A_df"):
        S64.apply_A_df(F)


def test_phase_times_count_the_outer_steps():
    """Phase timing of a refinement solve: one FP64 A x per FP64 outer residual,
    one double-float A x per provisional one, one FP32 A x (with the fused
    step length) and one preconditioner apply per inner iteration."""
    S = _solver(3, 3, 8, precision="tf32", refine=True)
    F = _cuda(synth.uniform(S.N, 11))
    S.solve(F, tol=1e-8, maxit=200)  # warm-up
    S.enable_timing(True)
    u, info = S.solve(F, tol=1e-8, maxit=200)
    ph = S.phase_times()
    S.enable_timing(False)
    it = info[0]
    assert it["status"] == "ok" and it["outer_df"] >= 1
    assert set(ph) == {"apply_A", "precond", "cg_vectors", "apply_A_f32", "apply_A_df"}
    assert ph["apply_A_df"][1] == it["outer_df"]
    assert ph["apply_A"][1] == it["outer"] - it["outer_df"]
    assert ph["apply_A_f32"][1] == it["iters"]
    assert ph["precond"][1] == it["iters"]  # one apply per outer step's start, one per further iteration
    assert all(v[0] >= 0.0 for v in ph.values())
