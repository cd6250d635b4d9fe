"""Pins for oracle.fd and oracle.solve (Sec. 4.2-4.3, Algorithm 1, Theorem 4, Table 1)."""
import os

import numpy as np
import pytest

from oracle.system import STProblem
from oracle.fd import FD
from oracle.solve import pcg, direct_solve

PI = np.pi
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("d,p,n_el,T", [(1, 2, 6, 1.0), (2, 3, 3, 1.0), (3, 4, 2, 0.5), (3, 6, 1, 1.0)])
def test_generalized_eigendecomposition(d, p, n_el, T):
    prob = STProblem(d, p, n_el, T)
    fd = FD(prob)
    for s, U, lam in zip(prob.space, fd.U, fd.lam):
        np.testing.assert_allclose(U.T @ s.M @ U, np.eye(s.n), atol=1e-13)
        np.testing.assert_allclose(U.T @ s.J @ U, np.diag(lam), atol=1e-9 * lam.max())
        assert np.all(np.diff(lam) >= 0)
    np.testing.assert_allclose(fd.U_t.T @ prob.time.M @ fd.U_t, np.eye(prob.n_t), atol=1e-13)


@pytest.mark.parametrize("d,p,n_el,T", [(1, 2, 5, 1.0), (1, 5, 3, 2.0), (2, 2, 4, 1.0),
                                        (2, 4, 2, 0.7), (3, 2, 3, 1.0), (3, 3, 2, 1.0)])
def test_fd_solve_is_explicit_inverse(d, p, n_el, T):
    prob = STProblem(d, p, n_el, T)
    fd = FD(prob)
    P = fd.explicit_P().toarray()
    Pinv = np.linalg.inv(P)
    rng = np.random.default_rng(3)
    for _ in range(3):
        r = rng.standard_normal(prob.N)
        np.testing.assert_allclose(fd.apply(r), Pinv @ r, atol=1e-10 * np.abs(Pinv @ r).max())
    r1, r2 = rng.standard_normal((2, prob.N))
    assert abs(r1 @ fd.apply(r2) - r2 @ fd.apply(r1)) < 1e-10 * abs(r1 @ fd.apply(r1))


def test_hat_pencil_equals_physical_pencil_at_T1():
    prob = STProblem(2, 3, 3, 1.0)
    r = np.random.default_rng(0).standard_normal(prob.N)
    np.testing.assert_allclose(FD(prob, "hat").apply(r), FD(prob).apply(r), rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("d,p", [(1, 2), (1, 4), (2, 2), (2, 3), (3, 2)])
def test_spectrum_of_preconditioned_matrix_is_bounded(d, p):
    """Theorem 4 on the unit cube: A(v,v) >= int (d_t v)^2 + (Lap v)^2 >= v^T P v and
    A(v,v) <= 2 ||v||_V0^2 <= 2d v^T P v, so 1 <= lambda(P^{-1} A) <= 2d for every mesh."""
    ns = {1: [4, 8, 16], 2: [2, 4, 6], 3: [1, 2, 3]}[d]
    bounds = []
    for n in ns:
        prob = STProblem(d, p, n, 1.0)
        A = prob.assemble_A_kron().toarray()
        P = FD(prob).explicit_P().toarray()
        ev = np.linalg.eigvals(np.linalg.solve(P, A)).real
        bounds.append((ev.min(), ev.max()))
        assert ev.min() >= 1 - 1e-9 and ev.max() <= 2 * d + 1e-9, bounds
    print(bounds)


def _cube_terms():
    s = lambda x: np.sin(PI * x)
    return [(1.0, np.cos, [s, s, s]), (3 * PI ** 2, np.sin, [s, s, s])]


def _table1():
    rows = {}
    for line in open(os.path.join(GOLDEN, "table1_cube_pcg_iterations.txt")):
        if line.startswith("#") or not line.strip():
            continue
        vals = line.split()
        rows[int(vals[0])] = [None if v == "*" else int(v) for v in vals[1:]]
    return rows


@pytest.mark.parametrize("n_sub", [8, 16, 32])
@pytest.mark.parametrize("p", [2, 3, 4, 5])
def test_table1_iteration_counts(n_sub, p):
    """P + CG on the cube, tol 1e-8, x0 = 0, u = sin sin sin sin(t) (Table 1)."""
    prob = STProblem(3, p, n_sub, 1.0)
    F = prob.load_separable(_cube_terms())
    _, it, _ = pcg(prob.apply_A_kron, FD(prob).apply, F, 1e-8, 100)
    assert it == _table1()[n_sub][p - 2]


@pytest.mark.parametrize("flexible", [False, True])
def test_pcg_matches_direct_solve(flexible):
    prob = STProblem(2, 3, 6, 1.0)
    A = prob.assemble_A_kron()
    F = np.random.default_rng(11).uniform(-1, 1, prob.N)
    x_ref = direct_solve(A, F)
    x, it, _ = pcg(lambda v: A @ v, FD(prob).apply, F, 1e-13, 200, flexible)
    np.testing.assert_allclose(x, x_ref, rtol=0, atol=1e-10 * np.abs(x_ref).max())
    np.testing.assert_allclose(prob.apply_A_kron(x), A @ x, rtol=1e-13, atol=1e-12)


@pytest.mark.parametrize("n_el,p", [(32, 4), (64, 3)])
def test_smallest_eigenvalues_to_high_relative_accuracy(n_el, p):
    """The eigenvalues that P^{-1} amplifies most, against 40-digit arithmetic."""
    mp = pytest.importorskip("mpmath")
    from oracle.fd import generalized_eig
    from oracle.spaces import Direction1D
    mp.mp.dps = 40
    s = Direction1D(n_el, p, "space")
    L = mp.cholesky(mp.matrix(s.M.tolist()))
    Li = L ** -1
    ref = sorted(float(e) for e in mp.eigsy(Li * mp.matrix(s.J.tolist()) * Li.T, eigvals_only=True))
    lam, _ = generalized_eig(s.J, s.M)
    np.testing.assert_allclose(lam[:5], ref[:5], rtol=1e-11)
    np.testing.assert_allclose(lam, ref, rtol=1e-10)
