"""Differentiable solve with a non-zero initial datum (Sec. 3.1 lifting).

Forward:  w = A^{-1} (F - G c0),  u = w + 1_{n_t} x c0   (G = e_T x L_s + m_t x J_s).
Backward: lam = A^{-1} g (adjoint solve with the same A and P, both
symmetric), dL/dF = lam, dL/dc0 = sum_t g[t, :] - G^T lam.
Every step runs in libstls.so; this file only orders the calls.
"""
import torch


class SolveFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, F, c0, solver, tol, maxit):
        rhs = solver.lifted_rhs(F, c0) if c0 is not None else F
        w, info = solver.solve(rhs.contiguous(), tol, maxit)
        ctx.solver, ctx.tol, ctx.maxit = solver, tol, maxit
        ctx.has_c0 = c0 is not None
        ctx.info = info
        if c0 is None:
            return w
        return solver.lift_add(w, c0)

    @staticmethod
    def backward(ctx, g):
        solver = ctx.solver
        g = g.contiguous()
        lam, _ = solver.solve(g, ctx.tol, ctx.maxit)
        dc0 = solver.lift_adjoint(g, lam) if ctx.has_c0 else None
        return lam, dc0, None, None, None
