"""Pins for oracle.spaces (Sec. 2.2, 4.1, 4.2, Remark of Sec. 4.4)."""
import numpy as np
import pytest

from oracle.spaces import Direction1D
from oracle.bspline import greville


@pytest.mark.parametrize("p", [2, 3, 4, 6])
def test_full_basis_identities(p):
    s = Direction1D(9, p, "space")
    one = np.ones(s.m)
    g = greville(s.knots, p)
    # M 1 = int b_i ; K 1 = 0 ; J 1 = 0 ; J g = 0 (g interpolates x, whose 2nd derivative is 0)
    ref = (s.knots[p + 1:] - s.knots[:s.m]) / (p + 1)
    np.testing.assert_allclose(s.M_full @ one, ref, rtol=1e-13)
    np.testing.assert_allclose(s.K_full @ one, 0.0, atol=1e-11)
    np.testing.assert_allclose(s.J_full @ one, 0.0, atol=1e-8)
    np.testing.assert_allclose(s.J_full @ g, 0.0, atol=1e-8)
    # K g = int b_i' * 1 = b_i(1) - b_i(0)
    e = np.zeros(s.m)
    e[0], e[-1] = -1.0, 1.0
    np.testing.assert_allclose(s.K_full @ g, e, atol=1e-11)
    for Mx in (s.M, s.K, s.J):
        np.testing.assert_allclose(Mx, Mx.T, atol=1e-12 * np.abs(Mx).max())
        assert np.linalg.eigvalsh(Mx).min() > 0
    # band of width 2p+1
    i, j = np.nonzero(np.abs(s.M_full) > 0)
    assert np.abs(i - j).max() == p


@pytest.mark.parametrize("p", [2, 3, 5])
def test_second_derivative_is_minus_stiffness_on_dirichlet_basis(p):
    s = Direction1D(7, p, "space")
    np.testing.assert_allclose(s.D2, -s.K, atol=1e-10 * np.abs(s.K).max())


@pytest.mark.parametrize("p", [1, 2, 4])
@pytest.mark.parametrize("T", [1.0, 0.37])
def test_time_end_term(p, T):
    tm = Direction1D(6, p, "time", length=T)
    # H + H^T = b(T) b(T)^T - b(0) b(0)^T = W on the reduced time basis
    np.testing.assert_allclose(tm.H + tm.H.T, tm.W, atol=1e-12)
    assert tm.W[-1, -1] == 1.0 and np.count_nonzero(tm.W) == 1


@pytest.mark.parametrize("T", [0.5, 2.0, 3.3])
def test_time_scaling_remark(T):
    hat = Direction1D(8, 3, "time", 1.0)
    phy = Direction1D(8, 3, "time", T)
    np.testing.assert_allclose(phy.K, hat.K / T, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(phy.M, hat.M * T, rtol=1e-12, atol=1e-14)


def test_sizes_match_reduced_space_counts():
    # Sec. 2.2: n_t = m_t - 1, n_s = m_s - 2 with m = n_el + p
    for n_el, p in [(16, 2), (64, 3), (32, 4), (48, 3)]:
        assert Direction1D(n_el, p, "space").n == n_el + p - 2
        assert Direction1D(n_el, p, "time").n == n_el + p - 1
