"""Pins for oracle.lifting (Sec. 3.1 lifting of a non-zero initial datum)."""
import numpy as np

from oracle.system import STProblem, kron_all
from oracle.lifting import solve_lifted, loss_and_grad
from oracle.solve import direct_solve


def _full_time_system(prob, f):
    """Least squares on the full time basis (first function included), by quadrature."""
    tm, sd = prob.time, prob.space
    all_t = np.arange(tm.m)
    dt = kron_all([s.B0[:, s.keep] for s in sd] + [tm.B1[:, all_t]])
    lap = 0
    for k in range(prob.d):
        mats = [s.B0[:, s.keep] for s in sd]
        mats[k] = sd[k].B2[:, sd[k].keep]
        lap = lap + kron_all(mats + [tm.B0[:, all_t]])
    w = kron_all([s.wq for s in sd] + [tm.wq])
    Phi = dt - lap
    grids = np.meshgrid(*([tm.xq] + [s.xq for s in sd[::-1]]), indexing="ij")
    xs = [g.ravel() for g in grids[1:][::-1]]
    fq = f(xs, grids[0].ravel())
    return Phi.T @ (w[:, None] * Phi), Phi.T @ (w * fq)


def test_lifting_equals_constrained_least_squares():
    prob = STProblem(2, 3, 3, 0.8, nq=6)
    f = lambda xs, t: np.sin(3 * xs[0]) * np.cos(xs[1]) * (1 + t)
    rng = np.random.default_rng(5)
    c0 = rng.standard_normal(prob.N_s)
    A_full, F_full = _full_time_system(prob, f)
    Ns = prob.N_s
    fixed, free = np.arange(Ns), np.arange(Ns, A_full.shape[0])
    u_free = np.linalg.solve(A_full[np.ix_(free, free)], F_full[free] - A_full[np.ix_(free, fixed)] @ c0)
    # reduced problem: same A and F restricted to the reduced basis
    A = prob.assemble_A_kron()
    np.testing.assert_allclose(A.toarray(), A_full[np.ix_(free, free)], atol=1e-11 * np.abs(A_full).max())
    u = solve_lifted(prob, A, F_full[free], c0)
    np.testing.assert_allclose(u, u_free, atol=1e-10 * np.abs(u_free).max())


def test_gradient_matches_central_differences():
    prob = STProblem(1, 3, 4, 1.0)
    A = prob.assemble_A_kron()
    rng = np.random.default_rng(9)
    F = rng.standard_normal(prob.N)
    c0 = rng.standard_normal(prob.N_s)
    ut = rng.standard_normal(prob.N)
    L, dF, dc0, _ = loss_and_grad(prob, A, F, c0, ut)
    h = 1e-6
    for _ in range(5):
        vF, vc = rng.standard_normal(prob.N), rng.standard_normal(prob.N_s)
        Lp = loss_and_grad(prob, A, F + h * vF, c0 + h * vc, ut)[0]
        Lm = loss_and_grad(prob, A, F - h * vF, c0 - h * vc, ut)[0]
        fd = (Lp - Lm) / (2 * h)
        an = dF @ vF + dc0 @ vc
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))
