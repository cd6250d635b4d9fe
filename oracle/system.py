"""Space-time system matrix A and load vector F (Sec. 3.2 and 4.1).

Oracle (test infrastructure).

Degrees of freedom are ordered colexicographically as in Sec. 4 (Eq.
kron_vec_multi): direction 1 runs fastest and time slowest, so a vector
reshapes in C order to an array of shape (n_t, n_d, ..., n_1), and a Kronecker
product of per-direction matrices is kron(W_t, W_d, ..., W_1).

Two independent constructions of A are provided:

* ``assemble_A_direct`` integrates the least-squares form of Eq. a-form,
  A_ij = int int (d_t B_j - Lap B_j)(d_t B_i - Lap B_i), by tensor Gauss
  quadrature of the basis functions themselves (tiny meshes only).
* ``assemble_A_kron`` builds A = K_t x M_s + M_t x J_s + W_t x L_s
  (Eq. A_kron) from the 1D matrices, with
  M_s = M_d x ... x M_1,  L_s = sum_k K_k x (M elsewhere), and
  J_s = int Lap B_i Lap B_j expanded over pairs of second derivatives:
  the k = l pairs give J_k, the k != l pairs give D2_k and D2_l^T in
  directions k and l, where D2[a,b] = int b''_a b_b.

Pinned by tests/test_oracle_system.py: the two constructions agree, A is
symmetric positive definite, A is coercive in the V0 norm (Lemma 2), and the
whole pipeline reproduces a solution that lies in the discrete space exactly.
"""
import numpy as np
import scipy.sparse as sp

from .spaces import Direction1D


def kron_all(mats):
    """kron(W_D, ..., W_1) for mats = [W_1, ..., W_D] (direction 1 fastest)."""
    out = mats[0]
    for W in mats[1:]:
        if sp.issparse(W) or sp.issparse(out):
            out = sp.kron(W, out, format="csr")
        else:
            out = np.kron(W, out)
    return out


def kron_vecs(vecs):
    """kron(v_D, ..., v_1) for vecs = [v_1, ..., v_D] (direction 1 fastest)."""
    out = np.ones(1)
    for v in vecs:
        out = np.kron(v, out)
    return out


class STProblem:
    """Heat equation on (0,1)^d x (0,T) with the reduced spline space of Sec. 2.2.

    ``n_el_s`` is an int (same for every direction) or a list of d ints.
    ``nq_extra`` adds Gauss points per element (for non-polynomial loads).
    """

    def __init__(self, d, p_s, n_el_s, T=1.0, p_t=None, n_el_t=None, nq=None):
        self.d = d
        self.p_s = p_s
        self.p_t = p_s if p_t is None else p_t
        if np.isscalar(n_el_s):
            n_el_s = [int(n_el_s)] * d
        self.n_el_s = list(n_el_s)
        self.n_el_t = self.n_el_s[0] if n_el_t is None else n_el_t
        self.T = float(T)
        self.space = [Direction1D(self.n_el_s[k], p_s, "space", 1.0, nq) for k in range(d)]
        self.time = Direction1D(self.n_el_t, self.p_t, "time", self.T, nq)
        self.n_s = [s.n for s in self.space]
        self.n_t = self.time.n
        self.N_s = int(np.prod(self.n_s))
        self.N = self.N_s * self.n_t
        self.shape = tuple([self.n_t] + self.n_s[::-1])   # C-order array shape

    # ---- spatial factors (Eq. A_kron) -------------------------------------------------
    def M_s(self):
        return kron_all([sp.csr_matrix(s.M) for s in self.space])

    def L_s(self):
        out = 0
        for k in range(self.d):
            mats = [sp.csr_matrix(s.M) for s in self.space]
            mats[k] = sp.csr_matrix(self.space[k].K)
            out = out + kron_all(mats)
        return sp.csr_matrix(out)

    def J_s(self):
        out = 0
        for k in range(self.d):
            for l in range(self.d):
                mats = [sp.csr_matrix(s.M) for s in self.space]
                if k == l:
                    mats[k] = sp.csr_matrix(self.space[k].J)
                else:
                    mats[k] = sp.csr_matrix(self.space[k].D2)
                    mats[l] = sp.csr_matrix(self.space[l].D2.T)
                out = out + kron_all(mats)
        return sp.csr_matrix(out)

    def assemble_A_kron(self):
        tm = self.time
        A = (sp.kron(sp.csr_matrix(tm.K), self.M_s())
             + sp.kron(sp.csr_matrix(tm.M), self.J_s())
             + sp.kron(sp.csr_matrix(tm.W), self.L_s()))
        return sp.csr_matrix(A)

    # ---- direct quadrature of Eq. a-form (tiny meshes) ----------------------------------
    def quad_operators(self):
        """Dense (d_t B_i)(q), (Lap B_i)(q) on the tensor Gauss grid, and its weights.

        Rows are grid points in colexicographic order, columns are the reduced
        basis functions; the tensor-product values come from Sec. 2.1
        (B_i(x, t) = prod_k b_{i_k}(x_k) b_{i_t}(t)).
        """
        tm, sd = self.time, self.space
        dt = kron_all([s.B0[:, s.keep] for s in sd] + [tm.B1[:, tm.keep]])
        lap = 0
        for k in range(self.d):
            mats = [s.B0[:, s.keep] for s in sd]
            mats[k] = sd[k].B2[:, sd[k].keep]
            lap = lap + kron_all(mats + [tm.B0[:, tm.keep]])
        w = kron_all([s.wq for s in sd] + [tm.wq])
        return dt, lap, w

    def _residual_operator(self):
        dt, lap, w = self.quad_operators()
        return dt - lap, w

    def assemble_A_direct(self, max_entries=6e7):
        nq = np.prod([len(s.wq) for s in self.space]) * len(self.time.wq)
        if nq * self.N > max_entries:
            raise ValueError("mesh too large for direct quadrature")
        Phi, w = self._residual_operator()
        return Phi.T @ (w[:, None] * Phi)

    def load_direct(self, f):
        """F_i = int int f (d_t B_i - Lap B_i) by tensor quadrature (tiny meshes).

        ``f(xs, t)`` takes a list of d coordinate arrays and a time array, all
        of the tensor quadrature grid, and returns f there.
        """
        Phi, w = self._residual_operator()
        grids = np.meshgrid(*([self.time.xq] + [s.xq for s in self.space[::-1]]), indexing="ij")
        t = grids[0].ravel()
        xs = [g.ravel() for g in grids[1:][::-1]]
        return Phi.T @ (w * f(xs, t))

    def load_separable(self, terms, nq=None):
        """F for f = sum_j c_j g_j(t) prod_k h_jk(x_k) (Sec. 3.2 definition of F).

        Each term is (c, g, [h_1, ..., h_d]).  The 1D integrals use ``nq``
        Gauss points per element (default p+5).  Uses
        int int f d_t B_i = (int g b'_it)(prod_k int h_k b_ik) and
        int int f Lap B_i = sum_k (int g b_it)(int h_k b''_ik)(prod_{l!=k} int h_l b_il).
        """
        fine_t = Direction1D(self.n_el_t, self.p_t, "time", self.T, nq or self.p_t + 5)
        fine_s = [Direction1D(self.n_el_s[k], self.p_s, "space", 1.0, nq or self.p_s + 5)
                  for k in range(self.d)]
        F = np.zeros(self.N)
        for c, g, hs in terms:
            gt = g(fine_t.xq) * fine_t.wq
            it0 = fine_t.B0[:, fine_t.keep].T @ gt
            it1 = fine_t.B1[:, fine_t.keep].T @ gt
            s0, s2 = [], []
            for k in range(self.d):
                hk = hs[k](fine_s[k].xq) * fine_s[k].wq
                s0.append(fine_s[k].B0[:, fine_s[k].keep].T @ hk)
                s2.append(fine_s[k].B2[:, fine_s[k].keep].T @ hk)
            F += c * kron_vecs(s0 + [it1])
            for k in range(self.d):
                vecs = list(s0)
                vecs[k] = s2[k]
                F -= c * kron_vecs(vecs + [it0])
        return F

    # ---- matrix-free Kronecker products (plain mode products) -----------------------------
    def to_tensor(self, v, batch=False):
        return v.reshape(((-1,) if batch else ()) + self.shape)

    def mode_product(self, X, W, k):
        """[X x_k W]: contract direction k (1..d space, d+1 time) with W[i, j] X[.., j, ..].

        X has C-order shape (n_t, n_d, ..., n_1) (optionally a leading batch axis).
        """
        axis = X.ndim - k if k <= self.d else X.ndim - self.d - 1
        Y = np.tensordot(W, X, axes=([1], [axis]))
        return np.moveaxis(Y, 0, axis)

    def apply_A_kron(self, x):
        """y = A x with A from Eq. A_kron, every Kronecker term applied by mode products."""
        X = x.reshape(self.shape)
        d, tm, sd = self.d, self.time, self.space
        Y = np.zeros_like(X)
        # K_t x M_s
        Z = X
        for k in range(d):
            Z = self.mode_product(Z, sd[k].M, k + 1)
        Y += self.mode_product(Z, tm.K, d + 1)
        # M_t x J_s
        for k in range(d):
            for l in range(d):
                Z = X
                for m in range(d):
                    if m == k and k == l:
                        W = sd[m].J
                    elif m == k:
                        W = sd[m].D2
                    elif m == l:
                        W = sd[m].D2.T
                    else:
                        W = sd[m].M
                    Z = self.mode_product(Z, W, m + 1)
                Y += self.mode_product(Z, tm.M, d + 1)
        # W_t x L_s
        for k in range(d):
            Z = X
            for m in range(d):
                Z = self.mode_product(Z, sd[m].K if m == k else sd[m].M, m + 1)
            Y += self.mode_product(Z, tm.W, d + 1)
        return Y.reshape(-1)


def apply_A_rows(prob, x, rows):
    """(A x)[rows] for sampled row indices, term by term from Eq. A_kron.

    Each row of a Kronecker term is the product of 1D rows, so an entry needs
    only the (2p+1)^(d+1) neighbours of the row's multi-index.  Used to check
    A x at sizes where the full product is too slow in plain numpy.
    """
    d, tm, sd = prob.d, prob.time, prob.space
    X = x.reshape(prob.shape)
    out = np.zeros(len(rows))
    terms = [([s.M for s in sd], tm.K), ]
    for k in range(d):
        for l in range(d):
            mats = [s.M for s in sd]
            if k == l:
                mats[k] = sd[k].J
            else:
                mats[k] = sd[k].D2
                mats[l] = sd[l].D2.T
            terms.append((mats, tm.M))
    for k in range(d):
        mats = [s.M for s in sd]
        mats[k] = sd[k].K
        terms.append((mats, tm.W))
    p_axes = [prob.p_t] + [prob.p_s] * d            # band half-widths per C-order axis
    for r, row in enumerate(rows):
        idx = np.unravel_index(row, prob.shape)   # (i_t, i_d, ..., i_1)
        win = [slice(max(0, i - pa), min(n, i + pa + 1)) for i, pa, n in zip(idx, p_axes, prob.shape)]
        Xw = X[tuple(win)]
        it, isp = idx[0], idx[1:][::-1]           # isp = (i_1, ..., i_d)
        wsp = win[1:][::-1]
        total = 0.0
        for mats, Tt in terms:
            Y = np.tensordot(Tt[it, win[0]], Xw, axes=([0], [0]))
            for k in range(d - 1, -1, -1):
                Y = np.tensordot(mats[k][isp[k], wsp[k]], Y, axes=([0], [0]))
            total += float(Y)
        out[r] = total
    return out
