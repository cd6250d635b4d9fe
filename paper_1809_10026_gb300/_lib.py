"""ctypes declarations of the C ABI in include/stls.h (argument marshalling only)."""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libstls.so")

STLS_OK, STLS_EINVAL, STLS_ENOMEM, STLS_ECUDA, STLS_ENOTCONV, STLS_EBREAKDOWN, STLS_ENONFINITE = range(7)
STATUS_NAMES = {0: "ok", 1: "invalid argument", 2: "out of memory", 3: "CUDA error",
                4: "not converged", 5: "breakdown", 6: "non-finite value"}
PRECISION = {"fp64": 0, "tf32": 1, "bf16": 2}
FACTOR = {"mass": 0, "stiff": 1, "bilap": 2, "eigvec": 3, "eigval": 4, "end": 5, "integral": 6,
          "geo_mass": 7, "geo_stiff": 8, "geo_bilap": 9, "geo_e": 10}
GEO_PRECOND = {"PG": 0, "Pbar": 1, "P": 2}

EXPORTS = ["stls_create", "stls_destroy", "stls_last_error", "stls_set_stream", "stls_sizes",
           "stls_apply_A", "stls_apply_A_df", "stls_apply_A_f32", "stls_apply_precond", "stls_solve", "stls_solve_host", "stls_apply_lift",
           "stls_lifted_rhs", "stls_lift_add", "stls_lift_adjoint", "stls_override_eigenvalues", "stls_residual_history", "stls_get_factor", "stls_host_factor", "stls_launch_count",
           "stls_enable_timing", "stls_phase_times", "stls_phase_times_n", "stls_apply_precond_noalloc", "stls_round_bf16",
           "stls_slab_spatial", "stls_slab_time", "stls_fd_spatial", "stls_fd_time_chunk", "stls_vec_dot",
           "stls_vec_axpby"]


class Params(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("p_s", ctypes.c_int), ("p_t", ctypes.c_int),
                ("n_el_s", ctypes.c_int * 3), ("n_el_t", ctypes.c_int), ("T", ctypes.c_double),
                ("precision", ctypes.c_int), ("flexible", ctypes.c_int), ("batch", ctypes.c_int),
                ("time_pencil", ctypes.c_int), ("refine", ctypes.c_int), ("inner_tol", ctypes.c_double),
                ("fp64_residuals", ctypes.c_int), ("geometry", ctypes.c_int), ("geo_a", ctypes.c_double * 3),
                ("geo_precond", ctypes.c_int)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("status", ctypes.c_int), ("rel_res", ctypes.c_double),
                ("true_rel_res", ctypes.c_double), ("outer", ctypes.c_int), ("outer_df", ctypes.c_int)]

    def as_dict(self):
        return {"iters": self.iters, "status": STATUS_NAMES.get(self.status, str(self.status)),
                "rel_res": self.rel_res, "true_rel_res": self.true_rel_res, "outer": self.outer,
                "outer_df": self.outer_df}


_lib = None


def load():
    """Load libstls.so; raises if the CUDA library has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libstls.so not found at %s: run __graft_entry__.build() or "
                          "python -m paper_1809_10026_gb300.build" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    vp, i = ctypes.c_void_p, ctypes.c_int
    for name in EXPORTS:
        getattr(lib, name).restype = ctypes.c_int
    lib.stls_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(Params), vp]
    lib.stls_destroy.argtypes = [vp]
    lib.stls_destroy.restype = None
    lib.stls_last_error.argtypes = [vp]
    lib.stls_last_error.restype = ctypes.c_char_p
    lib.stls_set_stream.argtypes = [vp, vp]
    lib.stls_sizes.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                               ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_int)]
    lib.stls_apply_A.argtypes = [vp, vp, vp]
    lib.stls_apply_A_df.argtypes = [vp, vp, vp]
    lib.stls_apply_A_f32.argtypes = [vp, vp, vp]
    lib.stls_apply_precond.argtypes = [vp, vp, vp]
    lib.stls_solve.argtypes = [vp, vp, vp, ctypes.c_double, i, ctypes.POINTER(SolveInfo)]
    lib.stls_solve_host.argtypes = [vp, vp, vp, ctypes.c_double, i, ctypes.POINTER(SolveInfo)]
    lib.stls_apply_lift.argtypes = [vp, vp, vp]
    lib.stls_lifted_rhs.argtypes = [vp, vp, vp, vp]
    lib.stls_lift_add.argtypes = [vp, vp, vp, vp]
    lib.stls_lift_adjoint.argtypes = [vp, vp, vp, vp]
    lib.stls_override_eigenvalues.argtypes = [vp, i, vp]
    lib.stls_residual_history.argtypes = [vp, i, vp, i, ctypes.POINTER(ctypes.c_int)]
    lib.stls_get_factor.argtypes = [vp, i, i, vp]
    lib.stls_host_factor.argtypes = [ctypes.POINTER(Params), i, i, vp]
    lib.stls_launch_count.argtypes = [vp]
    lib.stls_launch_count.restype = ctypes.c_longlong
    lib.stls_enable_timing.argtypes = [vp, i]
    lib.stls_phase_times.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)]
    lib.stls_phase_times_n.argtypes = [vp, i, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)]
    lib.stls_apply_precond_noalloc.argtypes = [i, ctypes.POINTER(ctypes.c_int), i, ctypes.POINTER(vp),
                                               ctypes.POINTER(vp), vp, vp, vp]
    lib.stls_round_bf16.argtypes = [vp, vp, ctypes.c_longlong, vp]
    ll = ctypes.c_longlong
    lib.stls_slab_spatial.argtypes = [vp, vp, ll, vp, vp, vp]
    lib.stls_slab_time.argtypes = [vp, vp, vp, i, i, i, i, vp, vp]
    lib.stls_fd_spatial.argtypes = [vp, vp, vp, ll, i]
    lib.stls_fd_time_chunk.argtypes = [vp, vp, vp, ll, ll]
    lib.stls_vec_dot.argtypes = [vp, vp, vp, ll, vp]
    lib.stls_vec_axpby.argtypes = [vp, vp, vp, vp, vp, ll]
    _lib = lib
    return lib


def make_params(d, p, n_el, T=1.0, precision="fp64", flexible=None, batch=1, p_t=None, n_el_t=None,
                time_pencil="physical", refine=False, inner_tol=0.0, fp64_residuals=False, geo_a=None,
                geo_precond="PG"):
    n_el_s = [int(n_el)] * d if isinstance(n_el, int) else [int(v) for v in n_el]
    if len(n_el_s) != d:
        raise ValueError("n_el must be an int or a list of d ints")
    prm = Params()
    prm.d = d
    prm.p_s = p
    prm.p_t = p if p_t is None else p_t
    for k in range(3):
        prm.n_el_s[k] = n_el_s[k] if k < d else 0
    prm.n_el_t = n_el_s[0] if n_el_t is None else n_el_t
    prm.T = float(T)
    prm.precision = PRECISION[precision]
    prm.flexible = int(precision != "fp64") if flexible is None else int(flexible)
    prm.batch = batch
    prm.time_pencil = {"physical": 0, "hat": 1}[time_pencil]
    prm.refine = int(bool(refine))
    prm.inner_tol = float(inner_tol)
    prm.fp64_residuals = int(bool(fp64_residuals))
    prm.geometry = 0 if geo_a is None else 1
    for k in range(3):
        prm.geo_a[k] = float(geo_a[k]) if geo_a is not None and k < len(geo_a) else 0.0
    prm.geo_precond = GEO_PRECOND[geo_precond]
    return prm
