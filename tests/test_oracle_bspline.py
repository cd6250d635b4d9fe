"""Pins for oracle.bspline (Sec. 2.1): library special case, partition of unity,
closed-form integrals and derivative identities."""
import numpy as np
import pytest
from scipy.interpolate import BSpline

from oracle.bspline import open_uniform_knots, basis, greville, gauss_legendre


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("n_el", [1, 3, 7])
def test_basis_matches_scipy(p, n_el):
    t = open_uniform_knots(n_el, p)
    m = n_el + p
    x = np.linspace(0.0, 1.0, 97, endpoint=False)[1:]
    for der in range(0, min(p, 2) + 1):
        ours = basis(t, p, x, der)
        for i in range(m):
            c = np.zeros(m)
            c[i] = 1.0
            ref = BSpline(t, c, p)(x, nu=der) if der else BSpline(t, c, p)(x)
            np.testing.assert_allclose(ours[:, i], ref, rtol=1e-12, atol=1e-10 * max(1, n_el ** der))


@pytest.mark.parametrize("p", [2, 3, 5])
def test_partition_of_unity_and_endpoints(p):
    t = open_uniform_knots(5, p)
    x = np.concatenate([np.linspace(0, 1, 41), [1.0]])
    B = basis(t, p, x)
    np.testing.assert_allclose(B.sum(axis=1), 1.0, atol=1e-14)
    np.testing.assert_allclose(basis(t, p, x, 1).sum(axis=1), 0.0, atol=1e-11)
    # open knots: interpolatory at both ends
    assert basis(t, p, [0.0])[0, 0] == 1.0 and basis(t, p, [1.0])[0, -1] == 1.0
    # Greville abscissae reproduce the identity: sum_i g_i b_i(x) = x
    np.testing.assert_allclose(B @ greville(t, p), x, atol=1e-14)


@pytest.mark.parametrize("p", [2, 4])
def test_integral_closed_form(p):
    # int b_i = (xi_{i+p+1} - xi_i) / (p + 1)
    t = open_uniform_knots(6, p, length=2.5)
    xq, wq = gauss_legendre(p + 1, t)
    ints = basis(t, p, xq).T @ wq
    ref = (t[p + 1:] - t[:len(t) - p - 1]) / (p + 1)
    np.testing.assert_allclose(ints, ref, rtol=1e-13)
