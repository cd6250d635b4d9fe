"""1D Galerkin matrices of the reduced spline bases (Sec. 2.2, 4.1, 4.2).

Oracle (test infrastructure).  For one parametric direction this module
assembles, by element-wise Gauss quadrature of the B-splines of
``oracle.bspline``, the full-basis matrices

    M[a,b] = int b_a b_b,   K[a,b] = int b'_a b'_b,   J[a,b] = int b''_a b''_b,
    D2[a,b] = int b''_a b_b,   H[a,b] = int b'_a b_b,

and restricts them to the reduced basis of Sec. 2.2: a space direction drops
the first and last function (homogeneous Dirichlet), the time direction drops
the first one (zero initial datum).  The time direction is integrated directly
on [0, T] with the knots scaled by T, so K_t and M_t are the physical matrices
of Eq. A_kron; the parametric (hat) matrices are the T = 1 case.

Pinned by tests/test_oracle_matrices.py: row sums against the closed-form
integral of a B-spline, K 1 = 0 and J g = 0 for the Greville abscissae g,
D2 = -K on the Dirichlet basis, H + H^T = W on the time basis, and the scaling
K_t = K_hat / T, M_t = T M_hat of the Remark in Sec. 4.4.
"""
import numpy as np

from .bspline import open_uniform_knots, basis, gauss_legendre


class Direction1D:
    """One parametric direction: knots, quadrature and reduced 1D matrices.

    kind = "space" keeps functions 2..m-1, kind = "time" keeps 2..m
    (1-based, Sec. 2.2).  ``nq`` Gauss points per element; the default p+1 is
    exact for every product of two degree-p splines and their derivatives.
    """

    def __init__(self, n_el, p, kind, length=1.0, nq=None):
        assert kind in ("space", "time")
        self.n_el, self.p, self.kind, self.length = n_el, p, kind, float(length)
        self.knots = open_uniform_knots(n_el, p, length)
        self.m = n_el + p
        self.nq = p + 1 if nq is None else nq
        self.xq, self.wq = gauss_legendre(self.nq, self.knots)
        self.B0 = basis(self.knots, p, self.xq, 0)
        self.B1 = basis(self.knots, p, self.xq, 1)
        self.B2 = basis(self.knots, p, self.xq, 2)
        W = self.wq[:, None]
        self.M_full = self.B0.T @ (W * self.B0)
        self.K_full = self.B1.T @ (W * self.B1)
        self.J_full = self.B2.T @ (W * self.B2)
        self.D2_full = self.B2.T @ (W * self.B0)
        self.H_full = self.B1.T @ (W * self.B0)
        if kind == "space":
            self.keep = np.arange(1, self.m - 1)
        else:
            self.keep = np.arange(1, self.m)
        self.n = len(self.keep)
        k = self.keep
        self.M = self.M_full[np.ix_(k, k)]
        self.K = self.K_full[np.ix_(k, k)]
        self.J = self.J_full[np.ix_(k, k)]
        self.D2 = self.D2_full[np.ix_(k, k)]
        self.H = self.H_full[np.ix_(k, k)]
        # values of the reduced basis at the right end (only the last is non-zero)
        self.end_values = basis(self.knots, p, [self.length], 0)[0, k]
        self.W = np.outer(self.end_values, self.end_values)
        # integrals of the reduced basis functions over the direction
        self.integrals = self.B0[:, k].T @ self.wq

    def eval(self, x, deriv=0):
        """Reduced-basis values (or derivatives) at points x: shape (len(x), n)."""
        return basis(self.knots, self.p, x, deriv)[:, self.keep]

    def project_coeffs(self, g):
        """Coefficients c of the reduced-basis interpolant of g at the Greville points.

        Used for the exact-reproduction pin: a function that lies in the
        reduced spline space is reproduced exactly by interpolation.
        """
        from .bspline import greville
        xg = greville(self.knots, self.p)[self.keep]
        return np.linalg.solve(self.eval(xg), g(xg))
