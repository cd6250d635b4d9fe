"""Preconditioner P and its fast-diagonalization solve (Sec. 4.2-4.3, Algorithm 1).

Oracle (test infrastructure).

P = K_t x M_s + M_t x Jt_s with M_s = M_d x ... x M_1 and
Jt_s = sum_k (J_k in direction k, M elsewhere)   (Eq. preconditioner).

The time pencil is the physical one, (M_t, K_t) integrated on [0, T]; by the
Remark of Sec. 4.4 this equals (T M_hat, K_hat / T), and for T = 1 it is the
parametric pencil printed in Eq. preconditioner.  ``time_pencil="hat"`` uses
the parametric pencil regardless of T.

Algorithm 1: generalized eigendecompositions J_k U_k = M_k U_k Lambda_k and
K_t U_t = M_t U_t Lambda_t with U^T M U = I (scipy.linalg.eigh), then
r~ = R x_1 U_1^T ... x_{d+1} U_t^T, q~ = r~ / (lambda_t[i_t] + sum_k lambda_k[i_k]),
s = Q~ x_1 U_1 ... x_{d+1} U_t.

LAPACK's generalized eigensolver is accurate to eps * ||M^{-1/2} J M^{-1/2}||
in absolute terms, which leaves the smallest eigenvalues (the ones P^{-1}
amplifies most) with relative errors near 1e-9 on 64-element meshes.  Each
eigenvalue is therefore taken as the Rayleigh quotient u^T J u / u^T M u of
its computed eigenvector, which is exact for an exact eigenvector and
accurate to the square of the eigenvector error otherwise.

Pinned by tests/test_oracle_fd.py: U^T M U = I and U^T J U = Lambda, the FD
solve equals the explicit inverse of the assembled P on tiny meshes, and the
spectrum of P^{-1} A stays in a mesh-independent interval (Theorem 4).
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .spaces import Direction1D
from .system import kron_all


def generalized_eig(J, M):
    """(lam, U) with J U = M U diag(lam), U^T M U = I, lam ascending (Rayleigh-refined)."""
    lam, U = sla.eigh(J, M)
    lam = np.einsum("ij,ik,kj->j", U, J, U) / np.einsum("ij,ik,kj->j", U, M, U)
    return lam, U


class FD:
    def __init__(self, prob, time_pencil="physical"):
        self.prob = prob
        self.lam, self.U = [], []
        for s in prob.space:
            lam, U = generalized_eig(s.J, s.M)
            self.lam.append(lam)
            self.U.append(U)
        if time_pencil == "physical":
            tm = prob.time
        else:
            tm = Direction1D(prob.n_el_t, prob.p_t, "time", 1.0)
        self.M_t, self.K_t = tm.M, tm.K
        self.lam_t, self.U_t = generalized_eig(tm.K, tm.M)

    def eig_tensor(self):
        """lambda_t[i_t] + sum_k lambda_k[i_k] as a C-order array (n_t, n_d, ..., n_1)."""
        prob = self.prob
        E = self.lam_t.reshape((-1,) + (1,) * prob.d)
        for k in range(prob.d):
            shape = [1] * (prob.d + 1)
            shape[prob.d - k] = prob.n_s[k]
            E = E + self.lam[k].reshape(shape)
        return E

    def apply(self, r):
        """s = P^{-1} r by Algorithm 1 (steps 2-4)."""
        prob = self.prob
        X = r.reshape(prob.shape)
        for k in range(prob.d):
            X = prob.mode_product(X, self.U[k].T, k + 1)
        X = prob.mode_product(X, self.U_t.T, prob.d + 1)
        X = X / self.eig_tensor()
        for k in range(prob.d):
            X = prob.mode_product(X, self.U[k], k + 1)
        X = prob.mode_product(X, self.U_t, prob.d + 1)
        return X.reshape(-1)

    def explicit_P(self):
        """P assembled from Kronecker products of the 1D matrices (Eq. preconditioner)."""
        prob = self.prob
        M_s = kron_all([sp.csr_matrix(s.M) for s in prob.space])
        Jt = 0
        for k in range(prob.d):
            mats = [sp.csr_matrix(s.M) for s in prob.space]
            mats[k] = sp.csr_matrix(prob.space[k].J)
            Jt = Jt + kron_all(mats)
        return sp.csr_matrix(sp.kron(sp.csr_matrix(self.K_t), M_s) + sp.kron(sp.csr_matrix(self.M_t), Jt))
