"""Non-zero initial datum by lifting (Sec. 3.1) and the adjoint gradient of a loss.

Oracle (test infrastructure).

With u(x, 0) = u0(x) = sum_i c0_i B_i(x) in the Dirichlet space spline space,
the lifting u0~(x, t) = u0(x) is constant in time, so f~ = f + Lap u0 and the
discrete unknown w = u - u0~ lies in V_{h,0}.  Testing the least-squares form
(Eq. a-form) with B_i(x) b_j(t):

    A(u0~, B_i b_j) = b_j(T) (L_s c0)_i + (int_0^T b_j) (J_s c0)_i,

so A w = F - G c0 with G = e_T x L_s + m_t x J_s (e_T the end values of the
time basis, m_t its integrals).  By the partition of unity the reduced
coefficients of u are w + 1_{n_t} x c0.

For L(u) = 0.5 ||u - u_target||^2 on the reduced coefficient vector:
g = u - u_target, lambda = A^{-1} g (A is symmetric), dL/dF = lambda and
dL/dc0 = sum_t g[t, :] - G^T lambda.

Pinned by tests/test_oracle_lifting.py: a brute-force least-squares solve on
the full time basis, with the coefficients of the first time function fixed
to c0, gives the same u; the gradient matches central differences.
"""
import numpy as np
import scipy.sparse as sp

from .solve import direct_solve


def lift_matrix(prob):
    e = prob.time.end_values
    m = prob.time.integrals
    return sp.csr_matrix(sp.kron(sp.csr_matrix(e[:, None]), prob.L_s())
                         + sp.kron(sp.csr_matrix(m[:, None]), prob.J_s()))


def solve_lifted(prob, A, F, c0):
    G = lift_matrix(prob)
    w = direct_solve(A, F - G @ c0)
    return w + np.kron(np.ones(prob.n_t), c0)


def loss_and_grad(prob, A, F, c0, u_target):
    G = lift_matrix(prob)
    u = solve_lifted(prob, A, F, c0)
    g = u - u_target
    lam = direct_solve(A, g)
    dF = lam
    dc0 = g.reshape(prob.n_t, prob.N_s).sum(axis=0) - G.T @ lam
    return 0.5 * g @ g, dF, dc0, u
