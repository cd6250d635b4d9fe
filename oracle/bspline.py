"""Univariate B-splines on open knot vectors (Sec. 2.1 of arXiv:1809.10026).

Oracle (test infrastructure).  Pinned by tests/test_oracle_bspline.py against
scipy.interpolate.BSpline (a library special case), the partition of unity and
the closed-form integrals of B-splines.
"""
import numpy as np


def open_uniform_knots(n_el, p, length=1.0):
    """Open knot vector with ``n_el`` equal elements on [0, length].

    Sec. 2.1: the first p+1 knots equal the left end, the last p+1 equal the
    right end.  There are m = n_el + p basis functions.
    """
    inner = [length * i / n_el for i in range(1, n_el)]
    return np.array([0.0] * (p + 1) + inner + [float(length)] * (p + 1))


def _safe_div(num, den):
    """num / den with the convention 0/0 = 0 used by the Cox-de Boor recursion."""
    out = np.zeros(np.broadcast(num, den).shape)
    den_b = np.broadcast_to(den, out.shape)
    num_b = np.broadcast_to(num, out.shape)
    nz = den_b != 0.0
    out[nz] = num_b[nz] / den_b[nz]
    return out


def basis(knots, q, x, deriv=0):
    """Values of all degree-q B-splines (or their ``deriv``-th derivative) at x.

    Returns an array of shape (len(x), len(knots) - q - 1); column i is b_{i,q}.

    Degree 0 is the indicator of [xi_i, xi_{i+1}); the right end of the knot
    vector is assigned to the last non-empty span so that the functions are
    continuous from the left at x = 1.  Degree q >= 1 is the Cox-de Boor
    recursion of Sec. 2.1, and derivatives use de Boor's formula
    b'_{i,q} = q ( b_{i,q-1} / (xi_{i+q} - xi_i) - b_{i+1,q-1} / (xi_{i+q+1} - xi_{i+1}) ),
    both with 0/0 = 0.
    """
    t = np.asarray(knots, dtype=float)
    x = np.atleast_1d(np.asarray(x, dtype=float))
    n_fun = len(t) - q - 1
    if q == 0:
        if deriv > 0:
            return np.zeros((len(x), n_fun))
        B = ((t[:-1][None, :] <= x[:, None]) & (x[:, None] < t[1:][None, :])).astype(float)
        last = max(i for i in range(len(t) - 1) if t[i] < t[i + 1])
        B[x == t[-1], :] = 0.0
        B[x == t[-1], last] = 1.0
        return B
    i = np.arange(n_fun)
    if deriv == 0:
        low = basis(t, q - 1, x, 0)
        left = _safe_div(x[:, None] - t[i][None, :], (t[i + q] - t[i])[None, :])
        right = _safe_div(t[i + q + 1][None, :] - x[:, None], (t[i + q + 1] - t[i + 1])[None, :])
        left = np.where((t[i + q] - t[i])[None, :] == 0.0, 0.0, left)
        right = np.where((t[i + q + 1] - t[i + 1])[None, :] == 0.0, 0.0, right)
        return left * low[:, i] + right * low[:, i + 1]
    low = basis(t, q - 1, x, deriv - 1)
    a = _safe_div(low[:, i], (t[i + q] - t[i])[None, :])
    b = _safe_div(low[:, i + 1], (t[i + q + 1] - t[i + 1])[None, :])
    return q * (a - b)


def greville(knots, p):
    """Greville abscissae (xi_{i+1} + ... + xi_{i+p}) / p of the degree-p basis."""
    t = np.asarray(knots, dtype=float)
    m = len(t) - p - 1
    return np.array([t[i + 1:i + p + 1].mean() for i in range(m)])


def gauss_legendre(n_el_pts, knots):
    """Element-wise Gauss-Legendre rule with ``n_el_pts`` points per non-empty span.

    Returns (points, weights) on [knots[0], knots[-1]].  numpy's leggauss
    supplies the reference rule on [-1, 1].
    """
    g, w = np.polynomial.legendre.leggauss(n_el_pts)
    t = np.asarray(knots, dtype=float)
    brk = np.unique(t)
    pts, wts = [], []
    for a, b in zip(brk[:-1], brk[1:]):
        pts.append(0.5 * (b - a) * g + 0.5 * (a + b))
        wts.append(0.5 * (b - a) * w)
    return np.concatenate(pts), np.concatenate(wts)
