"""Errors of a discrete solution in the V0, L2 and H1 norms (Sec. 3.2, 3.4, 5.1).

Oracle (test infrastructure).  The discrete solution is evaluated on a tensor
Gauss grid (``nq`` points per element) through the reduced 1D bases; the
exact solution is given by callables on the same grid.

V0 norm (Eq. norm_V0): ||v||^2 = int int (Lap v)^2 + (d_t v)^2.
L2 norm: int int v^2.  H1 norm (space-time): int int v^2 + |grad_x v|^2 + (d_t v)^2.
"""
import numpy as np

from .spaces import Direction1D


def _grid_eval(prob, c, mats):
    """Apply per-direction evaluation matrices to the coefficient tensor."""
    X = c.reshape(prob.shape)
    for k in range(prob.d):
        X = prob.mode_product(X, mats[k], k + 1)
    return prob.mode_product(X, mats[prob.d], prob.d + 1)


def errors(prob, c, exact, nq=None):
    """Relative errors {"V0", "L2", "H1"} of coefficient vector c against ``exact``.

    ``exact`` maps names "u", "ut", "lap", "grad" to callables f(xs, t) on the
    grid, with xs the list of d coordinate arrays (grad returns a list of d
    arrays).
    """
    d = prob.d
    nq = nq or prob.p_s + 3
    fs = [Direction1D(prob.n_el_s[k], prob.p_s, "space", 1.0, nq) for k in range(d)]
    ft = Direction1D(prob.n_el_t, prob.p_t, "time", prob.T, nq)
    E0 = [f.B0[:, f.keep] for f in fs] + [ft.B0[:, ft.keep]]
    uh = _grid_eval(prob, c, E0)
    uth = _grid_eval(prob, c, [f.B0[:, f.keep] for f in fs] + [ft.B1[:, ft.keep]])
    laph = 0
    gradh = []
    for k in range(d):
        m2 = list(E0)
        m2[k] = fs[k].B2[:, fs[k].keep]
        laph = laph + _grid_eval(prob, c, m2)
        m1 = list(E0)
        m1[k] = fs[k].B1[:, fs[k].keep]
        gradh.append(_grid_eval(prob, c, m1))
    grids = np.meshgrid(*([ft.xq] + [f.xq for f in fs[::-1]]), indexing="ij")
    t = grids[0]
    xs = grids[1:][::-1]
    w = ft.wq.reshape((-1,) + (1,) * d)
    for k in range(d):
        shape = [1] * (d + 1)
        shape[d - k] = -1
        w = w * fs[k].wq.reshape(shape)

    def integ(v):
        return float(np.sum(w * v))

    u, ut, lap, grad = exact["u"](xs, t), exact["ut"](xs, t), exact["lap"](xs, t), exact["grad"](xs, t)
    e, et, el = uh - u, uth - ut, laph - lap
    eg = [gh - g for gh, g in zip(gradh, grad)]
    out = {}
    out["V0"] = np.sqrt(integ(el ** 2 + et ** 2) / integ(lap ** 2 + ut ** 2))
    out["L2"] = np.sqrt(integ(e ** 2) / integ(u ** 2))
    h1 = integ(e ** 2 + et ** 2 + sum(g ** 2 for g in eg))
    h1u = integ(u ** 2 + ut ** 2 + sum(g ** 2 for g in grad))
    out["H1"] = np.sqrt(h1 / h1u)
    return out
