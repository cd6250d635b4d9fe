"""Least-squares system on a mapped cube and the geometry-aware preconditioner
P^G (Sec. 4.4: Eq. coefficients-c, Eq. coefficient-approx; App. A.3: the
separation-of-variables algorithm).

Oracle (test infrastructure).

Domain.  Omega = G((0,1)^d) with the separable map
    G(eta) = (g_1(eta_1), ..., g_d(eta_d)),  g_k(s) = s + a_k sin(2 pi s) / (2 pi),
|a_k| < 1: g_k(0) = 0, g_k(1) = 1 and g_k'(s) = 1 + a_k cos(2 pi s) > 0, so Omega
is the unit cube again, parametrized non-uniformly (the physical mesh is
stretched).  The basis functions are B_i = Bhat_i o G^{-1} for the reduced
tensor-product splines Bhat_i of Sec. 2.2; time is not mapped.

System.  A^G_ij = int_0^T int_Omega (d_t B_i - Lap B_i)(d_t B_j - Lap B_j) dx dt
(Eq. a-form on Omega), built two independent ways:
* ``assemble_direct``: tensor Gauss quadrature in (eta, t) of the form itself,
  with the physical Laplacian of every basis function from the general chain
  rule for a map (grad_x u = J^-T grad_eta u, Hess_x u = J^-T (Hess_eta u -
  sum_m (grad_x u)_m Hess_eta G_m) J^-1, Lap = trace), J and Hess G_m taken as
  full matrices from the map (tiny meshes only);
* ``assemble_kron``: for a separable map, Lap B = sum_k (L_k bhat) (other
  factors) with L_k b = (1/g_k') (b' / g_k')', |det J| = prod g_k', so
  A^G = K_t x M^w_s + M_t x J^w_s + W_t x L^w_s with the weighted 1D matrices
      M^w = int b b g',  K^w = int b' b' / g',  J^w = int (L b)(L b) g',
      E[a, b] = int (L b_a) b_b g'   (not symmetric),
  M^w_s = (x) M^w, L^w_s = sum_k K^w_k (M^w elsewhere) (the W_t term comes from
  integrating the cross terms by parts, as on the cube), and
  J^w_s = sum_k J^w_k + sum_{k != l} E_k (direction k) E_l^T (direction l)
  (M^w elsewhere).  On the cube (a = 0) E = -K and this is Eq. A_kron.

Preconditioner.  The coefficients of the leading terms of the form on the
parametric domain (Eq. coefficients-c):
  c_k = ||[J^-1]_{:,k}||^4 |det J| T (k = 1..d),  c_{d+1} = |det J| / T,
interpolated by their values at the element barycentres (tensors C^(k) over
the space-time elements), are approximated by products of univariate factors
(Eq. coefficient-approx) computed by the separation-of-variables algorithm
(``separate``), and
  Pbar^G = K^G_t x M^G_s + M^G_t x sum_k J^G_k (M^G elsewhere)
with [M^G_k]_ij = int mu_k b_i b_j, [J^G_k]_ij = int omega_k b''_i b''_j on
(0,1), [M^G_t]_ij = int mu_{d+1} b_i b_j, [K^G_t]_ij = int omega_{d+1} b'_i b'_j on
the parametric time interval (0,1).  Pbar^G keeps the Kronecker structure,
so Algorithm 1 applies it; P^G = D^{1/2} Pbar^G D^{1/2} with
D_ii = A^G_ii / Pbar^G_ii.

Reading of the algorithm (App. A.3).  Its mu-update builds, for direction k
and every other coefficient l, the ratio of C^(l) to its current product
approximation times mu^(k) (the estimate of mu^(k) that coefficient l gives,
since the approximation of c_l holds mu^(k) in direction k), takes the
element-wise min (Y) and max (Z) over l != k, and sets mu^(k)_j =
sqrt(min Y * max Z) over the slice i_k = j.  The printed listing indexes the
ratio with C^(k) and omega^(k); that reading does not decouple the two-variable
case as the text says it does (omega^(1), mu^(2) from C^(1); mu^(1),
omega^(2) from C^(2)), and this one does.

Pinned by tests/test_oracle_geometry.py: the two constructions of A^G agree,
the identity map gives the cube's A and P, the algorithm recovers exactly
separable tensors exactly, P^G applied by Algorithm 1 equals the explicit
inverse, and P^G reduces the PCG iteration count against P on a stretched
cube (the effect Table 2 shows on its curved domain).
"""
import numpy as np
import scipy.sparse as sp

from .bspline import basis, gauss_legendre
from .spaces import Direction1D
from .system import STProblem, kron_all
from .fd import generalized_eig


class StretchMap:
    """g_k(s) = s + a_k sin(2 pi s) / (2 pi) in each space direction."""

    def __init__(self, a):
        self.a = [float(v) for v in a]
        if any(abs(v) >= 1.0 for v in self.a):
            raise ValueError("|a_k| must be < 1")

    def g(self, k, s):
        return s + self.a[k] * np.sin(2 * np.pi * s) / (2 * np.pi)

    def dg(self, k, s):
        return 1.0 + self.a[k] * np.cos(2 * np.pi * s)

    def d2g(self, k, s):
        return -2 * np.pi * self.a[k] * np.sin(2 * np.pi * s)

    def jacobian(self, etas):
        """J (npts, d, d) and Hess G_m (npts, d, d, d) at points etas (npts, d), as
        full arrays (the direct assembly treats them as a general map's)."""
        npts, d = etas.shape
        J = np.zeros((npts, d, d))
        H = np.zeros((npts, d, d, d))
        for k in range(d):
            J[:, k, k] = self.dg(k, etas[:, k])
            H[:, k, k, k] = self.d2g(k, etas[:, k])
        return J, H


class MappedProblem:
    """The least-squares system of the heat equation on G((0,1)^d) x (0,T).

    ``nq``: Gauss points per element in space for the weighted
    (non-polynomial) integrands, default 2p + 6."""

    def __init__(self, d, p, n_el, a, T=1.0, nq=None):
        self.d, self.p, self.T = d, p, float(T)
        self.map = StretchMap(a)
        self.cube = STProblem(d, p, n_el, T)           # reduced spaces, time matrices, shapes
        self.N, self.shape = self.cube.N, self.cube.shape
        self.n_s, self.n_t = self.cube.n_s, self.cube.n_t
        self.nq = 2 * p + 6 if nq is None else nq
        self.fine = [Direction1D(n, p, "space", 1.0, self.nq) for n in self.cube.n_el_s]
        self.weighted = [self._weighted_1d(k) for k in range(d)]

    # ---- weighted 1D matrices of a separable map -------------------------------------------
    def _weighted_1d(self, k):
        s = self.fine[k]
        x, w = s.xq, s.wq
        g1, g2 = self.map.dg(k, x), self.map.d2g(k, x)
        B0, B1, B2 = (s.B0[:, s.keep], s.B1[:, s.keep], s.B2[:, s.keep])
        LB = B2 / g1[:, None] ** 2 - B1 * (g2 / g1 ** 3)[:, None]   # L_k b = (1/g')(b'/g')'
        W = w[:, None]
        return {"M": B0.T @ (W * g1[:, None] * B0),
                "K": B1.T @ (W / g1[:, None] * B1),
                "J": LB.T @ (W * g1[:, None] * LB),
                "E": LB.T @ (W * g1[:, None] * B0)}

    def assemble_kron(self):
        d, tm, wm = self.d, self.cube.time, self.weighted
        Mw = [sp.csr_matrix(w["M"]) for w in wm]
        Js, Ls = 0, 0
        for k in range(d):
            mats = list(Mw)
            mats[k] = sp.csr_matrix(wm[k]["K"])
            Ls = Ls + kron_all(mats)
            for l in range(d):
                mats = list(Mw)
                if k == l:
                    mats[k] = sp.csr_matrix(wm[k]["J"])
                else:
                    mats[k] = sp.csr_matrix(wm[k]["E"])
                    mats[l] = sp.csr_matrix(wm[l]["E"].T)
                Js = Js + kron_all(mats)
        Ms = kron_all(Mw)
        return sp.csr_matrix(sp.kron(sp.csr_matrix(tm.K), Ms) + sp.kron(sp.csr_matrix(tm.M), Js)
                             + sp.kron(sp.csr_matrix(tm.W), Ls))

    def apply_kron(self, x):
        """A^G x by mode products with the weighted 1D matrices (no assembly)."""
        pr, d, tm, wm = self.cube, self.d, self.cube.time, self.weighted
        X = x.reshape(self.shape)
        Y = np.zeros_like(X)

        def chain(mats):
            Z = X
            for m in range(d):
                Z = pr.mode_product(Z, mats[m], m + 1)
            return Z
        Mw = [w["M"] for w in wm]
        Y += pr.mode_product(chain(Mw), tm.K, d + 1)
        for k in range(d):
            for l in range(d):
                mats = list(Mw)
                if k == l:
                    mats[k] = wm[k]["J"]
                else:
                    mats[k] = wm[k]["E"]
                    mats[l] = wm[l]["E"].T
                Y += pr.mode_product(chain(mats), tm.M, d + 1)
        for k in range(d):
            mats = list(Mw)
            mats[k] = wm[k]["K"]
            Y += pr.mode_product(chain(mats), tm.W, d + 1)
        return Y.reshape(-1)

    # ---- direct quadrature of the form on Omega (tiny meshes) -------------------------------
    def _physical_residual_operator(self):
        """(d_t B_i - Lap_x B_i) at the space-time Gauss points, and the weights
        |det J| w, from the chain rule with full J and Hess G."""
        d, fine, tm = self.d, self.fine, self.cube.time
        # space points in colexicographic order (direction 1 fastest)
        grids = np.meshgrid(*[f.xq for f in fine[::-1]], indexing="ij")
        etas = np.stack([g.ravel() for g in grids[::-1]], axis=1)       # (nq_s, d)
        wsp = kron_all([f.wq for f in fine])
        J, HG = self.map.jacobian(etas)
        Jinv = np.linalg.inv(J)
        detJ = np.abs(np.linalg.det(J))
        # parametric derivatives of the spatial basis: values, gradient, Hessian
        V = [(f.B0[:, f.keep], f.B1[:, f.keep], f.B2[:, f.keep]) for f in fine]

        def tensor(orders):
            return kron_all([V[k][orders[k]] for k in range(d)])
        val = tensor([0] * d)
        grad = []
        for k in range(d):
            o = [0] * d
            o[k] = 1
            grad.append(tensor(o))
        hess = [[None] * d for _ in range(d)]
        for k in range(d):
            for l in range(d):
                o = [0] * d
                o[k] += 1
                o[l] += 1
                hess[k][l] = tensor(o)
        nb = val.shape[1]
        gphys = np.zeros((len(etas), nb, d))             # grad_x = J^-T grad_eta
        for i in range(d):
            for j in range(d):
                gphys[:, :, i] += Jinv[:, j, i][:, None] * grad[j]
        lap = np.zeros((len(etas), nb))
        for i in range(d):                               # trace of J^-T (H - sum_m g_m HG_m) J^-1
            for j in range(d):
                for l in range(d):
                    Hjl = hess[j][l] - sum(gphys[:, :, m] * HG[:, m, j, l][:, None] for m in range(d))
                    lap += Jinv[:, j, i][:, None] * Hjl * Jinv[:, l, i][:, None]
        # space-time: rows (t, space point), columns (t basis, space basis), C order
        bt0, bt1 = tm.B0[:, tm.keep], tm.B1[:, tm.keep]
        Phi = np.kron(bt1, val) - np.kron(bt0, lap)
        w = np.kron(tm.wq, wsp * detJ)
        return Phi, w

    def _space_time_points(self):
        """Physical space points (npts, d), time points, and the spatial basis values."""
        fine = self.fine
        grids = np.meshgrid(*[f.xq for f in fine[::-1]], indexing="ij")
        etas = np.stack([g.ravel() for g in grids[::-1]], axis=1)
        xs = np.stack([self.map.g(k, etas[:, k]) for k in range(self.d)], axis=1)
        val = kron_all([f.B0[:, f.keep] for f in fine])
        return xs, self.cube.time.xq, val

    def load_direct(self, f):
        """F_i = int int f (d_t B_i - Lap B_i) dx dt by the quadrature of
        assemble_direct; f(xs, t) with xs of shape (npts, d) physical points."""
        Phi, w = self._physical_residual_operator()
        xs, tq, _ = self._space_time_points()
        fv = np.concatenate([f(xs, np.full(len(xs), t)) for t in tq])
        return Phi.T @ (w * fv)

    def l2_error(self, c, u):
        """||u_h - u|| in L2(Omega x (0,T)), u_h = sum_i c_i B_i, u(xs, t) physical."""
        xs, tq, val = self._space_time_points()
        fine = self.fine
        etas_w = kron_all([f.wq for f in fine])
        J, _ = self.map.jacobian(np.stack([np.asarray(v) for v in
                                           np.meshgrid(*[f.xq for f in fine[::-1]], indexing="ij")[::-1]],
                                          axis=-1).reshape(-1, self.d))
        detJ = np.abs(np.linalg.det(J))
        bt = self.cube.time.B0[:, self.cube.time.keep]
        uh = (np.kron(bt, val) @ c)
        ue = np.concatenate([u(xs, np.full(len(xs), t)) for t in tq])
        w = np.kron(self.cube.time.wq, etas_w * detJ)
        return float(np.sqrt(np.sum(w * (uh - ue) ** 2)))

    def assemble_direct(self, max_entries=4e7):
        nq = np.prod([len(f.wq) for f in self.fine]) * len(self.cube.time.wq)
        if nq * self.N > max_entries:
            raise ValueError("mesh too large for direct quadrature")
        Phi, w = self._physical_residual_operator()
        return Phi.T @ (w[:, None] * Phi)

    # ---- the geometry-aware preconditioner --------------------------------------------------
    def coefficient_tensors(self):
        """C^(1..d+1): the coefficients c_k of Eq. coefficients-c at the
        barycentres of the space-time elements, shape (n_el_1, ..., n_el_d, n_el_t)
        (direction 1 first)."""
        d, T = self.d, self.T
        n_el = list(self.cube.n_el_s)
        mids = [(np.arange(n) + 0.5) / n for n in n_el]
        grids = np.meshgrid(*mids, indexing="ij")
        etas = np.stack([g.ravel() for g in grids], axis=1)
        J, _ = self.map.jacobian(etas)
        Jinv = np.linalg.inv(J)
        detJ = np.abs(np.linalg.det(J))
        ones_t = np.ones(self.cube.n_el_t)
        C = []
        for k in range(d):
            ck = np.linalg.norm(Jinv[:, :, k], axis=1) ** 4 * detJ * T
            C.append(np.multiply.outer(ck.reshape(n_el), ones_t))
        C.append(np.multiply.outer((detJ / T).reshape(n_el), ones_t))
        return C

    def preconditioner_factors(self, maxit=2):
        """Univariate factors (mu, omega) of Algorithm 2 and the 1D matrices of Pbar^G."""
        C = self.coefficient_tensors()
        mu, om = separate(C, maxit)
        d, p = self.d, self.p
        mats = []
        for k in range(d):
            s = self.cube.space[k]
            mats.append({"M": _elementwise(s, mu[k], 0), "J": _elementwise(s, om[k], 2)})
        th = Direction1D(self.cube.n_el_t, self.cube.p_t, "time", 1.0)
        tmat = {"M": _elementwise(th, mu[d], 0), "K": _elementwise(th, om[d], 1)}
        return mu, om, mats, tmat

    def preconditioner(self, maxit=2):
        """PG with apply(r) = (P^G)^{-1} r, explicit_Pbar(), D (the diagonal scaling)."""
        return GeometryFD(self, *self.preconditioner_factors(maxit)[2:])


def _elementwise(direction, weights, order):
    """int w b^(order)_i b^(order)_j for a weight constant on each element
    (p+1 Gauss points per element: exact)."""
    s = direction
    B = {0: s.B0, 1: s.B1, 2: s.B2}[order][:, s.keep]
    nq = s.nq
    wel = np.repeat(np.asarray(weights, dtype=float), nq)
    return B.T @ ((s.wq * wel)[:, None] * B)


def separate(C, maxit=2):
    """Algorithm 2 (App. A.3): positive vectors mu^(k), omega^(k) with
    C^(k) ~ mu^(1) ... omega^(k) ... mu^(D) (D = len(C) directions), the
    min/max ratio in each slice driven towards 1 in the log sense."""
    D = len(C)
    shape = C[0].shape
    mu = [np.ones(n) for n in shape]
    om = [np.ones(n) for n in shape]

    def expand(v, axis):
        s = [1] * D
        s[axis] = -1
        return v.reshape(s)

    def prod_mu(skip):
        P = np.ones(shape)
        for l in range(D):
            if l not in skip:
                P = P * expand(mu[l], l)
        return P

    def slice_minmax(Ymin, Zmax, axis):
        other = tuple(a for a in range(D) if a != axis)
        return np.sqrt(Ymin.min(axis=other) * Zmax.max(axis=other))

    for _ in range(maxit):
        for k in range(D):
            V = C[k] / prod_mu({k})
            om[k] = slice_minmax(V, V, k)
        for k in range(D):
            Ws = []
            for l in range(D):
                if l == k:
                    continue
                approx_l = prod_mu({l}) * expand(om[l], l)
                Ws.append(C[l] / approx_l * expand(mu[k], k))
            Y = np.minimum.reduce(Ws)
            Z = np.maximum.reduce(Ws)
            mu[k] = slice_minmax(Y, Z, k)
    return mu, om


class GeometryFD:
    """(P^G)^{-1} = D^{-1/2} Pbar^{-1} D^{-1/2} with Pbar^{-1} by Algorithm 1."""

    def __init__(self, prob, smats, tmat):
        self.prob, self.smats, self.tmat = prob, smats, tmat
        self.lam, self.U = [], []
        for m in smats:
            lam, U = generalized_eig(m["J"], m["M"])
            self.lam.append(lam)
            self.U.append(U)
        self.lam_t, self.U_t = generalized_eig(tmat["K"], tmat["M"])
        self.D = self.diag_A() / self.diag_Pbar()

    def diag_A(self):
        """diag(A^G) from the 1D diagonals of the Kronecker form."""
        pr = self.prob
        d, tm, wm = pr.d, pr.cube.time, pr.weighted
        dM = [np.diag(w["M"]) for w in wm]
        out = np.kron(np.diag(tm.K), kron_all(dM))
        for k in range(d):
            for l in range(d):
                v = list(dM)
                if k == l:
                    v[k] = np.diag(wm[k]["J"])
                else:
                    v[k] = np.diag(wm[k]["E"])
                    v[l] = np.diag(wm[l]["E"])
                out = out + np.kron(np.diag(tm.M), kron_all(v))
        for k in range(d):
            v = list(dM)
            v[k] = np.diag(wm[k]["K"])
            out = out + np.kron(np.diag(tm.W), kron_all(v))
        return out

    def diag_Pbar(self):
        d = self.prob.d
        dM = [np.diag(m["M"]) for m in self.smats]
        out = np.kron(np.diag(self.tmat["K"]), kron_all(dM))
        for k in range(d):
            v = list(dM)
            v[k] = np.diag(self.smats[k]["J"])
            out = out + np.kron(np.diag(self.tmat["M"]), kron_all(v))
        return out

    def explicit_Pbar(self):
        d = self.prob.d
        Ms = kron_all([sp.csr_matrix(m["M"]) for m in self.smats])
        Jt = 0
        for k in range(d):
            mats = [sp.csr_matrix(m["M"]) for m in self.smats]
            mats[k] = sp.csr_matrix(self.smats[k]["J"])
            Jt = Jt + kron_all(mats)
        return sp.csr_matrix(sp.kron(sp.csr_matrix(self.tmat["K"]), Ms) + sp.kron(sp.csr_matrix(self.tmat["M"]), Jt))

    def apply_Pbar_inverse(self, r):
        pr = self.prob.cube
        d = pr.d
        X = r.reshape(pr.shape)
        for k in range(d):
            X = pr.mode_product(X, self.U[k].T, k + 1)
        X = pr.mode_product(X, self.U_t.T, d + 1)
        E = self.lam_t.reshape((-1,) + (1,) * d)
        for k in range(d):
            s = [1] * (d + 1)
            s[d - k] = -1
            E = E + self.lam[k].reshape(s)
        X = X / E
        for k in range(d):
            X = pr.mode_product(X, self.U[k], k + 1)
        X = pr.mode_product(X, self.U_t, d + 1)
        return X.reshape(-1)

    def apply(self, r):
        s = 1.0 / np.sqrt(self.D)
        return s * self.apply_Pbar_inverse(s * r)
