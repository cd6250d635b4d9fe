"""GB300 space-time least-squares heat-equation solver (arXiv:1809.10026).

Thin Python binding over the C ABI of include/stls.h: every step of the
solver runs in libstls.so (CUDA, sm_103a).  PyTorch provides device memory
and streams.  There is no CPU fallback: constructing a Solver without the
compiled library or without a CUDA device raises.
"""
import ctypes

import numpy as np

from . import _lib
from ._lib import FACTOR, make_params

__all__ = ["Solver", "SolveFn", "host_factor", "make_params", "round_bf16"]


def _check(rc, ctx=None):
    if rc != _lib.STLS_OK:
        lib = _lib.load()
        msg = lib.stls_last_error(ctx).decode()
        raise RuntimeError("stls error %d (%s): %s" % (rc, _lib.STATUS_NAMES.get(rc, "?"), msg))


def host_factor(which, direction, d, p, n_el, **kw):
    """A 1D factor computed by the library's host setup (no GPU needed)."""
    prm = make_params(d, p, n_el, **kw)
    lib = _lib.load()
    n_s = [n + prm.p_s - 2 for n in list(prm.n_el_s)[:d]]
    n = n_s[direction] if direction < d else prm.n_el_t + prm.p_t - 1
    size = n if FACTOR[which] in (4, 5, 6) else n * n
    out = np.zeros(size)
    rc = lib.stls_host_factor(ctypes.byref(prm), FACTOR[which], direction,
                              out.ctypes.data_as(ctypes.c_void_p))
    _check(rc)
    return out if size == n else out.reshape(n, n)


def round_bf16(x):
    """FP64(BF16(FP32(x))) elementwise on the GPU (stls_round_bf16): the operand
    rounding of the BF16 preconditioner.  x: CUDA float64 tensor."""
    import torch
    if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.float64):
        raise TypeError("round_bf16 expects a CUDA float64 tensor")
    x = x.contiguous()
    y = torch.empty_like(x)
    lib = _lib.load()
    rc = lib.stls_round_bf16(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), x.numel(),
                             ctypes.c_void_p(torch.cuda.current_stream(x.device).cuda_stream))
    _check(rc)
    return y


class Solver:
    """Solver context for (0,1)^d x (0,T) with degree p splines and n_el elements.

    precision: "fp64" or the mixed forms "tf32" / "bf16" (tensor-core FD
    mode products with FP32 accumulation; FP32 division by the eigenvalue
    sums; with refine=False every CG vector, A x and inner product in FP64).
    refine=True (mixed forms) solves by iterative refinement: FP64 residuals
    F - A u and corrections, inner FP32 flexible CG.
    geo_a (FP64 only): stretch amplitudes a_k of the parametrization
    g_k(s) = s + a_k sin(2 pi s) / (2 pi) of the cube (Sec. 4.4 setting);
    geo_precond "PG" (P^G with the diagonal scaling), "Pbar" or "P" (the
    parametric cube's P).  Vectors are float64 CUDA tensors of
    shape (batch, N) or (N,) for batch 1, in colexicographic order
    (direction 1 fastest, time slowest).
    """

    def __init__(self, d, p, n_el, T=1.0, precision="fp64", flexible=None, batch=1, p_t=None,
                 n_el_t=None, time_pencil="physical", device=None, refine=False, inner_tol=0.0,
                 fp64_residuals=False, geo_a=None, geo_precond="PG"):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("stls.Solver needs a CUDA device (no CPU fallback)")
        self.torch = torch
        self.device = torch.device("cuda" if device is None else device)
        self.lib = _lib.load()
        self.params = make_params(d, p, n_el, T, precision, flexible, batch, p_t, n_el_t, time_pencil,
                                  refine, inner_tol, fp64_residuals, geo_a, geo_precond)
        self.ctx = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            stream = torch.cuda.current_stream(self.device).cuda_stream
            rc = self.lib.stls_create(ctypes.byref(self.ctx), ctypes.byref(self.params),
                                      ctypes.c_void_p(stream))
        if rc != _lib.STLS_OK:
            raise RuntimeError("stls_create failed (%d): %s" % (rc, self.lib.stls_last_error(None).decode()))
        n_s = (ctypes.c_int * 3)()
        n_t, n_dof, b = ctypes.c_int(), ctypes.c_longlong(), ctypes.c_int()
        self.lib.stls_sizes(self.ctx, n_s, ctypes.byref(n_t), ctypes.byref(n_dof), ctypes.byref(b))
        self.d = d
        self.n_s = [n_s[k] for k in range(d)]
        self.n_t = n_t.value
        self.N = n_dof.value
        self.N_s = self.N // self.n_t
        self.batch = b.value
        self.precision = precision

    # ---- marshalling ------------------------------------------------------------------
    def _stream(self):
        s = self.torch.cuda.current_stream(self.device).cuda_stream
        self.lib.stls_set_stream(self.ctx, ctypes.c_void_p(s))

    def _vec(self, x, n, name):
        t = self.torch
        if not isinstance(x, t.Tensor) or x.dtype != t.float64 or x.device.type != "cuda":
            raise TypeError("%s must be a float64 CUDA tensor" % name)
        if x.numel() != self.batch * n:
            raise ValueError("%s must have batch * %d = %d entries, got %d" % (name, n, self.batch * n, x.numel()))
        return x.contiguous()

    def _out(self, like_shape, n):
        return self.torch.empty((self.batch, n) if self.batch > 1 else (n,), dtype=self.torch.float64,
                                device=self.device)

    @staticmethod
    def _ptr(x):
        return ctypes.c_void_p(x.data_ptr())

    # ---- operators -------------------------------------------------------------------
    def apply_A(self, x, out=None):
        x = self._vec(x, self.N, "x")
        y = self._out(x.shape, self.N) if out is None else out
        self._stream()
        _check(self.lib.stls_apply_A(self.ctx, self._ptr(x), self._ptr(y)), self.ctx)
        return y

    def apply_A_df(self, x, out=None):
        """A x in double-float arithmetic (FP32 pairs), as the refinement form's
        provisional outer residuals use it; refinement contexts only."""
        x = self._vec(x, self.N, "x")
        y = self._out(x.shape, self.N) if out is None else out
        self._stream()
        _check(self.lib.stls_apply_A_df(self.ctx, self._ptr(x), self._ptr(y)), self.ctx)
        return y

    def apply_A_f32(self, x, out=None):
        """A x in FP32 arithmetic, the operator of the refinement form's inner
        solves; x and the result are float32 CUDA tensors; refinement contexts only."""
        t = self.torch
        if not isinstance(x, t.Tensor) or x.dtype != t.float32 or x.device.type != "cuda":
            raise TypeError("x must be a float32 CUDA tensor")
        if x.numel() != self.batch * self.N:
            raise ValueError("x must have batch * %d = %d entries, got %d" % (self.N, self.batch * self.N, x.numel()))
        x = x.contiguous()
        y = t.empty((self.batch, self.N) if self.batch > 1 else (self.N,), dtype=t.float32,
                    device=self.device) if out is None else out
        self._stream()
        _check(self.lib.stls_apply_A_f32(self.ctx, self._ptr(x), self._ptr(y)), self.ctx)
        return y

    def apply_precond(self, r, out=None):
        r = self._vec(r, self.N, "r")
        z = self._out(r.shape, self.N) if out is None else out
        self._stream()
        _check(self.lib.stls_apply_precond(self.ctx, self._ptr(r), self._ptr(z)), self.ctx)
        return z

    def solve(self, F, tol=1e-8, maxit=500, out=None, check=True):
        F = self._vec(F, self.N, "F")
        u = self._out(F.shape, self.N) if out is None else out
        info = (_lib.SolveInfo * self.batch)()
        self._stream()
        rc = self.lib.stls_solve(self.ctx, self._ptr(F), self._ptr(u), float(tol), int(maxit), info)
        infos = [info[b].as_dict() for b in range(self.batch)]
        if check and rc not in (_lib.STLS_OK,):
            _check(rc, self.ctx)
        return u, infos

    def solve_host(self, F, tol=1e-8, maxit=500, u=None):
        """F, u: float64 numpy arrays (pinned memory is faster) of batch * N entries."""
        F = np.ascontiguousarray(F, dtype=np.float64)
        if F.size != self.batch * self.N:
            raise ValueError("F has the wrong size")
        u = np.empty_like(F) if u is None else u
        info = (_lib.SolveInfo * self.batch)()
        self._stream()
        rc = self.lib.stls_solve_host(self.ctx, F.ctypes.data_as(ctypes.c_void_p),
                                      u.ctypes.data_as(ctypes.c_void_p), float(tol), int(maxit), info)
        _check(rc, self.ctx)
        return u, [info[b].as_dict() for b in range(self.batch)]

    def solve_host_ptr(self, F_ptr, u_ptr, tol=1e-8, maxit=500):
        """Same as solve_host with raw host pointers (e.g. pinned torch tensors)."""
        info = (_lib.SolveInfo * self.batch)()
        self._stream()
        rc = self.lib.stls_solve_host(self.ctx, ctypes.c_void_p(F_ptr), ctypes.c_void_p(u_ptr),
                                      float(tol), int(maxit), info)
        _check(rc, self.ctx)
        return [info[b].as_dict() for b in range(self.batch)]

    def apply_lift(self, c0):
        c0 = self._vec(c0, self.N_s, "c0")
        y = self._out(c0.shape, self.N)
        self._stream()
        _check(self.lib.stls_apply_lift(self.ctx, self._ptr(c0), self._ptr(y)), self.ctx)
        return y

    def lifted_rhs(self, F, c0):
        """F - G c0: the right-hand side of the problem with initial datum c0."""
        F = self._vec(F, self.N, "F")
        c0 = self._vec(c0, self.N_s, "c0")
        rhs = self._out(F.shape, self.N)
        self._stream()
        _check(self.lib.stls_lifted_rhs(self.ctx, self._ptr(F), self._ptr(c0), self._ptr(rhs)), self.ctx)
        return rhs

    def lift_add(self, w, c0):
        """u = w + 1_{n_t} x c0: the solution of the lifted problem from its correction w."""
        w = self._vec(w, self.N, "w")
        c0 = self._vec(c0, self.N_s, "c0")
        u = self._out(w.shape, self.N)
        self._stream()
        _check(self.lib.stls_lift_add(self.ctx, self._ptr(w), self._ptr(c0), self._ptr(u)), self.ctx)
        return u

    def lift_adjoint(self, g, lam):
        g = self._vec(g, self.N, "g")
        lam = self._vec(lam, self.N, "lam")
        dc0 = self._out(g.shape, self.N_s)
        self._stream()
        _check(self.lib.stls_lift_adjoint(self.ctx, self._ptr(g), self._ptr(lam), self._ptr(dc0)), self.ctx)
        return dc0

    def factor(self, which, direction):
        n = self.n_s[direction] if direction < self.d else self.n_t
        size = n if FACTOR[which] in (4, 5, 6) else n * n
        out = np.zeros(size)
        _check(self.lib.stls_get_factor(self.ctx, FACTOR[which], direction,
                                        out.ctypes.data_as(ctypes.c_void_p)), self.ctx)
        return out if size == n else out.reshape(n, n)

    def residual_history(self, b=0):
        """||r_k|| / ||F|| of right-hand side b in the last solve (stls_residual_history)."""
        n = ctypes.c_int()
        _check(self.lib.stls_residual_history(self.ctx, int(b), None, 0, ctypes.byref(n)), self.ctx)
        out = np.zeros(n.value)
        _check(self.lib.stls_residual_history(self.ctx, int(b), out.ctypes.data_as(ctypes.c_void_p), n.value,
                                              ctypes.byref(n)), self.ctx)
        return out

    def override_eigenvalues(self, direction, lam):
        """Testing hook: the FP64 preconditioner divides by these eigenvalues of
        `direction` from now on (stls_override_eigenvalues)."""
        n = self.n_s[direction] if direction < self.d else self.n_t
        lam = np.ascontiguousarray(lam, dtype=np.float64)
        if lam.size != n:
            raise ValueError("expected %d eigenvalues" % n)
        _check(self.lib.stls_override_eigenvalues(self.ctx, int(direction), lam.ctypes.data_as(ctypes.c_void_p)),
               self.ctx)

    def launch_count(self):
        return int(self.lib.stls_launch_count(self.ctx))

    def enable_timing(self, on=True):
        _check(self.lib.stls_enable_timing(self.ctx, int(on)), self.ctx)

    def phase_times(self):
        names = ["apply_A", "precond", "cg_vectors", "apply_A_f32", "apply_A_df"]
        ms = (ctypes.c_double * len(names))()
        cnt = (ctypes.c_longlong * len(names))()
        _check(self.lib.stls_phase_times_n(self.ctx, len(names), ms, cnt), self.ctx)
        return {names[i]: (ms[i], cnt[i]) for i in range(len(names))}

    def close(self):
        if getattr(self, "ctx", None) and self.ctx.value:
            self.lib.stls_destroy(self.ctx)
            self.ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


from .autograd import SolveFn  # noqa: E402
