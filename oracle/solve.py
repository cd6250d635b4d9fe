"""Direct solve and preconditioned CG (Sec. 4.2, Sec. 5: tolerance, zero initial guess).

Oracle (test infrastructure).

``pcg`` is the textbook preconditioned conjugate gradient method started from
x0 = 0 and stopped when the recursively updated residual satisfies
||r_k||_2 / ||F||_2 <= tol.  With ``flexible=True`` the direction update uses
the Polak-Ribiere form beta = (z_{k+1}, r_{k+1} - r_k) / (z_k, r_k) of
flexible CG (Notay, SIAM J. Sci. Comput. 22 (2000)), which tolerates a
preconditioner that is not exactly linear (such as one applied in reduced
precision).  Pinned by the iteration counts of Table 1 and by agreement with
the direct solve.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def direct_solve(A, F):
    if sp.issparse(A):
        return spla.spsolve(sp.csc_matrix(A), F)
    return np.linalg.solve(A, F)


def pcg(apply_A, apply_P, F, tol, maxit, flexible=False):
    """Returns (x, iterations, history of relative residuals)."""
    x = np.zeros_like(F)
    r = F.copy()
    nF = np.linalg.norm(F)
    hist = [1.0]
    if nF == 0.0:
        return x, 0, hist
    z = apply_P(r)
    p = z.copy()
    rz = r @ z
    for it in range(1, maxit + 1):
        q = apply_A(p)
        alpha = rz / (p @ q)
        x += alpha * p
        r -= alpha * q
        rel = np.linalg.norm(r) / nF
        hist.append(rel)
        if rel <= tol:
            return x, it, hist
        z = apply_P(r)
        rz_new = r @ z
        beta = (-alpha * (z @ q) / rz) if flexible else (rz_new / rz)
        rz = rz_new
        p = z + beta * p
    return x, maxit, hist
