"""Pins for oracle.system (Sec. 3.2, 4.1): Eq. a-form vs Eq. A_kron, SPD,
coercivity (Lemma 2), exact reproduction of a discrete solution, the load
vector, and the a-priori convergence rates (Theorem 3, Sec. 5.1)."""
import numpy as np
import pytest

from oracle.system import STProblem
from oracle.solve import direct_solve
from oracle.norms import errors

PI = np.pi


@pytest.mark.parametrize("d,p,n_el,T", [(1, 2, 3, 1.0), (1, 3, 4, 0.6), (1, 5, 2, 1.0),
                                        (2, 2, 3, 1.0), (2, 3, 2, 1.7), (3, 2, 2, 1.0), (3, 3, 1, 0.8)])
def test_a_form_equals_kronecker_form(d, p, n_el, T):
    prob = STProblem(d, p, n_el, T)
    A1 = prob.assemble_A_direct()
    A2 = prob.assemble_A_kron().toarray()
    scale = np.abs(A1).max()
    np.testing.assert_allclose(A2, A1, atol=1e-12 * scale)
    # symmetric positive definite
    np.testing.assert_allclose(A1, A1.T, atol=1e-13 * scale)
    np.linalg.cholesky(A1)


def test_anisotropic_kronecker_form():
    prob = STProblem(2, 3, [2, 3], T=1.3, p_t=2, n_el_t=4)
    np.testing.assert_allclose(prob.assemble_A_kron().toarray(), prob.assemble_A_direct(),
                               atol=1e-12 * np.abs(prob.assemble_A_direct()).max())


@pytest.mark.parametrize("d,p,n_el", [(1, 3, 4), (2, 2, 3)])
def test_coercivity_in_V0_norm(d, p, n_el):
    prob = STProblem(d, p, n_el, 1.0)
    A = prob.assemble_A_kron()
    dt, lap, w = prob.quad_operators()
    rng = np.random.default_rng(7)
    for _ in range(20):
        v = rng.standard_normal(prob.N)
        v0 = np.sum(w * (dt @ v) ** 2) + np.sum(w * (lap @ v) ** 2)
        assert v @ (A @ v) >= v0 * (1 - 1e-12)
        # the gap is exactly the end-time gradient term of Eq. equivalent_A
        assert v @ (A @ v) - v0 >= -1e-10 * v0


def _exact_terms(d):
    q = lambda x: x * (1 - x)
    one = lambda x: np.ones_like(x)
    terms = [(1.0, lambda t: np.ones_like(t), [q] * d)]
    for k in range(d):
        hs = [q] * d
        hs[k] = one
        terms.append((2.0, lambda t: t, hs))
    return terms


@pytest.mark.parametrize("d,p,n_el,T", [(1, 2, 5, 1.0), (1, 4, 3, 0.7), (2, 3, 3, 1.0), (3, 2, 2, 1.3)])
def test_exact_reproduction(d, p, n_el, T):
    """u = prod_k x_k(1-x_k) * t lies in V_{h,0}, so least squares returns it exactly."""
    prob = STProblem(d, p, n_el, T)
    cx = [s.project_coeffs(lambda x: x * (1 - x)) for s in prob.space]
    ct = prob.time.project_coeffs(lambda t: t)
    u_ref = ct
    for c in cx[::-1]:
        u_ref = np.kron(u_ref, c)
    F = prob.load_separable(_exact_terms(d))
    u = direct_solve(prob.assemble_A_kron(), F)
    np.testing.assert_allclose(u, u_ref, atol=1e-11 * np.abs(u_ref).max())


def test_load_vector_separable_vs_direct():
    prob = STProblem(2, 3, 3, 0.9, nq=9)
    terms = [(PI, lambda t: np.cos(t), [lambda x: np.sin(PI * x), lambda y: np.sin(2 * PI * y)]),
             (-0.3, lambda t: t ** 2, [lambda x: np.exp(x), lambda y: y])]

    def f(xs, t):
        return sum(c * g(t) * h[0](xs[0]) * h[1](xs[1]) for c, g, h in terms)

    F1 = prob.load_separable(terms, nq=9)
    F2 = prob.load_direct(f)
    np.testing.assert_allclose(F1, F2, atol=1e-12 * np.abs(F2).max())


def sin_solution_1d():
    terms = [(PI, lambda t: np.cos(PI * t), [lambda x: np.sin(PI * x)]),
             (PI ** 2, lambda t: np.sin(PI * t), [lambda x: np.sin(PI * x)])]
    exact = {
        "u": lambda xs, t: np.sin(PI * xs[0]) * np.sin(PI * t),
        "ut": lambda xs, t: PI * np.sin(PI * xs[0]) * np.cos(PI * t),
        "lap": lambda xs, t: -PI ** 2 * np.sin(PI * xs[0]) * np.sin(PI * t),
        "grad": lambda xs, t: [PI * np.cos(PI * xs[0]) * np.sin(PI * t)],
    }
    return terms, exact


@pytest.mark.parametrize("p,norm,rate", [(2, "V0", 1), (3, "V0", 2), (4, "V0", 3),
                                         (2, "H1", 2), (3, "H1", 3),
                                         (3, "L2", 4), (4, "L2", 5), (2, "L2", 2)])
def test_convergence_rates(p, norm, rate):
    """V0: h^(p-1) (Theorem 3); H1: h^p and L2: h^(p+1) for p >= 3 (Sec. 5.1);
    p = 2 L2 is suboptimal (Sec. 5.1) -- read here as the fourth-order-problem rate h^2."""
    terms, exact = sin_solution_1d()
    errs = []
    ns = [8, 16, 32] if p < 4 else [4, 8, 16]
    for n in ns:
        prob = STProblem(1, p, n, 1.0)
        u = direct_solve(prob.assemble_A_kron(), prob.load_separable(terms))
        errs.append(errors(prob, u, exact)[norm])
    observed = np.log2(errs[-2] / errs[-1])
    assert abs(observed - rate) < 0.35, (errs, observed)


def sin_solution_2d():
    """u = sin(pi x) sin(pi y) sin(t) (the two-dimensional manufactured solution)."""
    s = lambda x: np.sin(PI * x)
    terms = [(1.0, np.cos, [s, s]), (2 * PI ** 2, np.sin, [s, s])]
    exact = {
        "u": lambda xs, t: np.sin(PI * xs[0]) * np.sin(PI * xs[1]) * np.sin(t),
        "ut": lambda xs, t: np.sin(PI * xs[0]) * np.sin(PI * xs[1]) * np.cos(t),
        "lap": lambda xs, t: -2 * PI ** 2 * np.sin(PI * xs[0]) * np.sin(PI * xs[1]) * np.sin(t),
        "grad": lambda xs, t: [PI * np.cos(PI * xs[0]) * np.sin(PI * xs[1]) * np.sin(t),
                               PI * np.sin(PI * xs[0]) * np.cos(PI * xs[1]) * np.sin(t)],
    }
    return terms, exact


@pytest.mark.parametrize("p", [2, 3])
def test_convergence_rates_2d(p):
    """Two space dimensions: V0 h^(p-1) (Theorem 3), H1 h^p, L2 h^(p+1) for
    p = 3 and h^2 for p = 2 (Sec. 5.1), on n_el = 4, 8, 16."""
    terms, exact = sin_solution_2d()
    errs = []
    for n in (4, 8, 16):
        prob = STProblem(2, p, n, 1.0)
        u = direct_solve(prob.assemble_A_kron(), prob.load_separable(terms))
        errs.append(errors(prob, u, exact))
    expected = {"V0": p - 1, "H1": p, "L2": p + 1 if p >= 3 else 2}
    for norm, rate in expected.items():
        observed = np.log2(errs[-2][norm] / errs[-1][norm])
        assert abs(observed - rate) < 0.35, (norm, observed)


@pytest.mark.parametrize("p_t", [2, 3])
def test_unbalanced_degrees_gain_one_order(p_t):
    """Spatial degree p_s = p_t + 1: the V0 error converges as h^(p_t), one
    order above the h^(p_t - 1) of p_s = p_t (Sec. 5.1, unbalanced degrees)."""
    terms, exact = sin_solution_1d()

    def v0_rate(p_s):
        errs = []
        for n in (8, 16, 32):
            prob = STProblem(1, p_s, n, 1.0, p_t=p_t)
            u = direct_solve(prob.assemble_A_kron(), prob.load_separable(terms))
            errs.append(errors(prob, u, exact)["V0"])
        return np.log2(errs[-2] / errs[-1])

    unbalanced, balanced = v0_rate(p_t + 1), v0_rate(p_t)
    assert abs(unbalanced - p_t) < 0.35, unbalanced
    assert abs(balanced - (p_t - 1)) < 0.35, balanced


@pytest.mark.parametrize("d,p,n_el", [(1, 2, 5), (2, 3, 4), (3, 2, 3)])
def test_sampled_rows_of_A(d, p, n_el):
    from oracle.system import apply_A_rows
    prob = STProblem(d, p, n_el, 0.8)
    x = np.random.default_rng(0).standard_normal(prob.N)
    y = prob.assemble_A_kron() @ x
    np.testing.assert_allclose(apply_A_rows(prob, x, np.arange(prob.N)), y, atol=1e-13 * np.abs(y).max())
    np.testing.assert_allclose(prob.apply_A_kron(x), y, atol=1e-13 * np.abs(y).max())
