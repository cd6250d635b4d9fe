/*
 * stls.h -- C ABI of the GB300 space-time least-squares heat-equation solver.
 *
 * Problem (Montardini, Negri, Sangalli, Tani, arXiv:1809.10026):
 *   heat equation d_t u - Lap u = f on (0,1)^d x (0,T), u = 0 on the spatial
 *   boundary, u = 0 at t = 0 (Sec. 3.1, Eq. heat_eq), discretized by the
 *   least-squares method of Sec. 3.3 with tensor-product B-splines of degree
 *   p_s in space and p_t in time on uniform open knot vectors (Sec. 2).
 *   The unknowns are the coefficients of the reduced basis of Sec. 2.2: space
 *   directions drop their first and last B-spline, time drops its first one,
 *   so n_s,k = n_el,k + p_s - 2, n_t = n_el,t + p_t - 1, N = n_t * prod n_s,k.
 *
 * Layout of every vector argument: FP64, colexicographic order of Sec. 4
 *   (Eq. kron_vec_multi): direction 1 fastest, time slowest; a batch of B
 *   right-hand sides is B consecutive vectors of N entries (row-major
 *   (B, n_t, n_d, ..., n_1)).  Device pointers must be 8-byte aligned and may
 *   not overlap unless a function says otherwise.
 *
 * Ownership: the caller owns every buffer it passes in; the context owns its
 *   1D factors and its workspace, allocated once in stls_create.  No call
 *   other than stls_create allocates device memory.
 *
 * Streams: every call is ordered on the CUDA stream given to stls_create or
 *   stls_set_stream.  stls_apply_* are asynchronous; stls_solve* synchronize
 *   with the host to test convergence.
 *
 * Errors: every int-returning call returns STLS_OK (0) or a stls_status code,
 *   and stls_last_error(ctx) describes the last failure.  Invalid sizes or
 *   parameters are rejected before any launch.
 */
#ifndef STLS_H
#define STLS_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct stls_ctx stls_ctx;

enum stls_status {
  STLS_OK = 0,
  STLS_EINVAL = 1,      /* invalid parameter, size or pointer */
  STLS_ENOMEM = 2,      /* device or host allocation failed (stls_create only) */
  STLS_ECUDA = 3,       /* a CUDA runtime call or kernel launch failed */
  STLS_ENOTCONV = 4,    /* CG reached maxit before the tolerance */
  STLS_EBREAKDOWN = 5,  /* CG breakdown: (p, A p) <= 0 or (z, r) <= 0 */
  STLS_ENONFINITE = 6   /* a NaN or Inf appeared in the data or the iteration */
};

/* Arithmetic of the preconditioner (Algorithm 1) and of the solve.
 * STLS_FP64: FP64 throughout.
 * STLS_MIXED_TF32 / STLS_MIXED_BF16: the mode products of steps 2 and 4 run
 * on the tensor cores with TF32 / BF16 operands and FP32 accumulation; the
 * tensors between products are stored in FP32 rounded to TF32 (TF32 form)
 * or in BF16.  The eigenvalues are computed in FP64 on the host.  The
 * division of step 3 runs in FP32: its divisor is the FP32 sum of lambda_t
 * (rounded once from FP64) and of the spatial sum sum_k lambda_k[i_k]
 * (formed in FP64 and rounded once), and the quotient is rounded to the
 * operand format before the backward products; the FP32 division's error, a
 * few units in the last FP32 place, is three orders of magnitude below that
 * rounding.  The input r is rounded to FP32 and then to the operand format;
 * z leaves as the FP32 accumulator (widened exactly to FP64 when the
 * vectors are FP64).
 * Where the rest of the solve runs in FP64 depends on `refine`: with
 * refine = 0 (strict form), A x, the residual, every CG vector and every
 * inner product are FP64; with refine = 1 only the outer residual F - A u
 * (provisional steps in double-float arithmetic, see `refine`) and the
 * correction of u are FP64, and the inner solve is FP32 as described there.
 * The mixed forms should be used with flexible = 1. */
enum stls_precision { STLS_FP64 = 0, STLS_MIXED_TF32 = 1, STLS_MIXED_BF16 = 2 };

typedef struct {
  int d;            /* spatial dimension, 1..3 */
  int p_s;          /* spline degree in space, >= 2 (C^1 splines, Assumption 2) */
  int p_t;          /* spline degree in time, >= 1 */
  int n_el_s[3];    /* elements per spatial direction (first d entries), >= 1 */
  int n_el_t;       /* elements in time, >= 1 */
  double T;         /* final time, > 0 */
  int precision;    /* enum stls_precision */
  int flexible;     /* 1: flexible CG (Polak-Ribiere beta), 0: standard PCG */
  int batch;        /* right-hand sides per call, 1..1024 */
  int time_pencil;  /* 0: time pencil (M_t, K_t) on [0,T]; 1: parametric (T = 1)
                       pencil of Eq. preconditioner.  Equal when T = 1. */
  int refine;       /* mixed forms only.  0: flexible CG in FP64 with the
                       tensor-core preconditioner.  1: iterative refinement:
                       an outer loop computes the residual r = F - A u in FP64
                       and corrects u (in FP64) with an inner flexible CG in
                       FP32: FP32 vectors x, r, p, q, z, FP32 A p, the
                       tensor-core preconditioner on FP32 input and output,
                       and inner products accumulated per thread in
                       compensated FP32 (TwoProd and TwoSum, about twice the
                       FP32 precision) and across threads in FP64; it reduces
                       its scaled residual by inner_tol.  With d = 2, 3 an outer step whose
                       predicted residual ||r|| max(inner residual, 4e-4) exceeds
                       both 100 tol and 1e-8 takes a provisional residual with
                       the double-float A x (stls_apply_A_df); the FP64 residual
                       decides every convergence test. */
  double inner_tol; /* relative tolerance of the inner solves.  0: adaptive:
                       the reduction R = tol ||F|| / ||r|| still needed is split
                       over K = ceil(log R / log 1e-3) outer steps, inner
                       tolerance R^(1/K) clamped to [1e-4, 0.1]; at most 400
                       inner iterations per outer step */
  int fp64_residuals; /* refine = 1 only.  0: provisional double-float outer
                       residuals as described under refine; 1: every outer
                       residual F - A u in FP64 */
  /* Parametrization of the spatial domain (Sec. 4.4).  0: the unit cube with
     the identity map.  1: the unit cube parametrized by the separable map
     G(eta)_k = g_k(eta_k) = eta_k + geo_a[k] sin(2 pi eta_k) / (2 pi), a
     non-uniformly stretched mesh of the same domain; the unknowns are the
     coefficients of the mapped splines Bhat_i o G^{-1}, and A is the
     least-squares matrix of Eq. a-form on the mapped basis (weighted 1D
     factors; every 1D integral by 2p_s + 6 Gauss points per element).
     geometry = 1 needs precision = STLS_FP64 and offers stls_apply_A,
     stls_apply_precond and stls_solve (no lifting calls). */
  int geometry;
  double geo_a[3];    /* geometry = 1: stretch amplitudes, |geo_a[k]| < 1 (first d entries) */
  int geo_precond;    /* geometry = 1: preconditioner.  0: P^G = D^{1/2} Pbar^G D^{1/2}
                         of Sec. 4.4 (coefficients of Eq. coefficients-c at the
                         element barycentres, univariate factors by the
                         separation-of-variables algorithm of App. A.3 with two
                         sweeps, D = diag(A) / diag(Pbar^G)); 1: Pbar^G alone;
                         2: P of the parametric cube (the geometry ignored) */
} stls_params;

typedef struct {
  int iters;            /* CG iterations performed (inner iterations when refine = 1) */
  int status;           /* STLS_OK, STLS_ENOTCONV, STLS_EBREAKDOWN or STLS_ENONFINITE */
  double rel_res;       /* ||r_k|| / ||F|| of the residual the stopping test used:
                           recursively updated (refine = 0) or F - A u in FP64 (refine = 1) */
  double true_rel_res;  /* ||F - A u|| / ||F|| recomputed in FP64 at exit */
  int outer;            /* outer steps of the refinement loop, each ended by a residual
                           evaluation (0 if refine = 0) */
  int outer_df;         /* of those, provisional residuals in double-float arithmetic
                           (stls_apply_A_df); the FP64 residual confirmed the last one */
} stls_solve_info;

/* Create a solver context: builds the 1D Galerkin matrices (Sec. 4.1-4.2) and
 * the generalized eigendecompositions of Algorithm 1, step 1, on the host in
 * FP64, uploads them and allocates the workspace for `batch` right-hand
 * sides.  `cuda_stream` is a cudaStream_t (NULL = legacy default stream).
 * On failure *out is NULL and the return code says why.  Calls on one
 * context must not overlap (one host thread at a time); contexts of any
 * sizes may coexist in a process and be used one after another. */
int stls_create(stls_ctx **out, const stls_params *prm, void *cuda_stream);

/* Release everything the context owns.  NULL is accepted. */
void stls_destroy(stls_ctx *ctx);

/* Text of the last error on this context ("" if none).  With ctx == NULL,
 * the last failure of a context-free call on the calling thread
 * (stls_create, stls_host_factor, stls_round_bf16,
 * stls_apply_precond_noalloc). */
const char *stls_last_error(const stls_ctx *ctx);

/* Change the stream used by later calls. */
int stls_set_stream(stls_ctx *ctx, void *cuda_stream);

/* Sizes: n_s[0..d-1] reduced spatial sizes, *n_t, *n_dof = N (per RHS),
 * *batch.  Any pointer may be NULL. */
int stls_sizes(const stls_ctx *ctx, int *n_s, int *n_t, long long *n_dof, int *batch);

/* y = A x for the batch (Eq. A_kron: A = K_t x M_s + M_t x J_s + W_t x L_s),
 * matrix-free by banded mode products in FP64.  x, y: device, B x N. */
int stls_apply_A(stls_ctx *ctx, const double *x, double *y);

/* y = A x as stls_apply_A, in double-float arithmetic: every FP64 value is
 * carried as the unevaluated sum of two FP32 values (about 48 significant
 * bits) and every product and sum runs on the FP32 pipe.  This is the
 * operator of the refinement form's provisional outer residuals (the FP64
 * residual confirms convergence).  Accurate while x, A x and the
 * intermediate products stay inside the FP32 normal range (about 1e-38 to
 * 3e38 in magnitude).  x, y: device, B x N, must not overlap.  Errors:
 * STLS_EINVAL unless the context has refine = 1, d = 2 or 3 and degrees
 * 1..6 (the fused A x). */
int stls_apply_A_df(stls_ctx *ctx, const double *x, double *y);

/* y = A x in FP32 arithmetic: the operator of the refinement form's inner
 * flexible CG (Sec. 4.2 on the system of Eq. A_kron), with the bands rounded
 * once to FP32 and every product and sum an FP32 operation (fused
 * multiply-add, fixed order).  x, y: device, B x N FP32, must not overlap.
 * Errors: STLS_EINVAL unless the context has refine = 1. */
int stls_apply_A_f32(stls_ctx *ctx, const float *x, float *y);

/* z = P^{-1} r for the batch by fast diagonalization (Eq. preconditioner,
 * Algorithm 1, steps 2-4) in the context's precision.  r, z: device, B x N;
 * r == z is allowed. */
int stls_apply_precond(stls_ctx *ctx, const double *r, double *z);

/* Operand rounding of the BF16 preconditioner (the mixed form of Algorithm 1,
 * step 2): y[i] = x[i] rounded to FP32, then to BF16, both to nearest with
 * ties to even, returned exactly as FP64.  This is how the BF16 form rounds
 * its FP64 input r before the first mode product.  x, y: device, n entries
 * (x == y allowed), n >= 0; ordered on `cuda_stream` (NULL = legacy default
 * stream), asynchronous.  Needs no context.  Errors: STLS_EINVAL (n < 0, NULL
 * pointer with n > 0), STLS_ECUDA; text via stls_last_error(NULL). */
int stls_round_bf16(const double *x, double *y, long long n, void *cuda_stream);

/* Solve A u = F for the batch by (flexible) preconditioned CG from u = 0,
 * stopping each right-hand side when ||r_k|| / ||F|| <= tol (Sec. 5: tolerance
 * on the relative residual, zero initial guess).  With refine = 1, maxit bounds
 * the total inner iterations and the test uses the FP64 residual F - A u.
 * F, u: device, B x N.
 * info: host array of B entries (may be NULL).  Returns STLS_OK if every
 * right-hand side converged, else the first non-OK per-RHS status. */
int stls_solve(stls_ctx *ctx, const double *F, double *u, double tol, int maxit,
               stls_solve_info *info);

/* As stls_solve, with F and u in HOST memory (B x N each): copies F to the
 * device, solves, copies u back, and returns when u_host holds the result.
 * Pinned host memory gives the fastest copies.  In the refinement form the
 * copy of u runs on a second stream of the context while the FP64 residual
 * that may confirm convergence is computed (u no longer changes then), and is
 * repeated if a further outer step changes u; u_host may therefore be written
 * more than once during the call. */
int stls_solve_host(stls_ctx *ctx, const double *F_host, double *u_host, double tol,
                    int maxit, stls_solve_info *info);

/* Lifting of a non-zero initial datum u0 = sum_i c0_i B_i(x) (Sec. 3.1):
 * y = G c0 with G = e_T x L_s + m_t x J_s, where e_T holds the time basis at
 * t = T and m_t its integrals over (0,T).  The discrete problem with initial
 * datum u0 is A w = F - G c0, and u = w + 1_{n_t} x c0.
 * c0: device, B x N_s; y: device, B x N. */
int stls_apply_lift(stls_ctx *ctx, const double *c0, double *y);

/* Right-hand side of the lifted problem: rhs = F - G c0 (G as for
 * stls_apply_lift).  F, rhs: device, B x N; c0: device, B x N_s; rhs must
 * not overlap F or c0.  Uses the context's workspace (stream-ordered like
 * every call on the context). */
int stls_lifted_rhs(stls_ctx *ctx, const double *F, const double *c0, double *rhs);

/* Solution of the lifted problem from its correction: u = w + 1_{n_t} x c0,
 * i.e. u[b, t, :] = w[b, t, :] + c0[b, :] for every time index t.
 * w, u: device, B x N; c0: device, B x N_s; u must not overlap w or c0. */
int stls_lift_add(stls_ctx *ctx, const double *w, const double *c0, double *u);

/* Adjoint of the lifted solve for a loss L(u): given g = dL/du and
 * lam = A^{-1} g, writes dc0 = sum_t g[t, :] - G^T lam (device, B x N_s). */
int stls_lift_adjoint(stls_ctx *ctx, const double *g, const double *lam, double *dc0);

/* Factor ids for stls_get_factor / stls_host_factor. */
enum stls_factor {
  STLS_F_MASS = 0,      /* n x n  M_k (space) / M_t (time, on [0,T]) */
  STLS_F_STIFF = 1,     /* n x n  K_k / K_t */
  STLS_F_BILAP = 2,     /* n x n  J_k = int b''_i b''_j (space only) */
  STLS_F_EIGVEC = 3,    /* n x n  U of the preconditioner pencil, row-major */
  STLS_F_EIGVAL = 4,    /* n      Lambda of the preconditioner pencil, ascending */
  STLS_F_END = 5,       /* n      time basis at t = T (time only) */
  STLS_F_INTEGRAL = 6,  /* n      integrals of the reduced basis functions */
  /* geometry = 1, space directions: the weighted factors of A (g = g_k) */
  STLS_F_GEO_MASS = 7,  /* n x n  int b_i b_j g' */
  STLS_F_GEO_STIFF = 8, /* n x n  int b'_i b'_j / g' */
  STLS_F_GEO_BILAP = 9, /* n x n  int (L b_i)(L b_j) g',  L b = (1/g') (b' / g')' */
  STLS_F_GEO_E = 10     /* n x n  int (L b_i) b_j g'  (not symmetric) */
};
/* With geometry = 1, STLS_F_EIGVEC / STLS_F_EIGVAL are those of the pencils of
 * the context's preconditioner (Pbar^G unless geo_precond = 2). */

/* Copy a 1D factor of direction `dir` (0..d-1 space, d = time) to host
 * memory.  Matrices are row-major. */
int stls_get_factor(const stls_ctx *ctx, int which, int dir, double *host_out);

/* Relative residuals ||r_k|| / ||F|| of right-hand side b (0..B-1) in the
 * last solve on this context, as the convergence test saw them: entry 0 is
 * the initial residual (1, or 0 when F = 0), then one entry per CG iteration
 * (refine = 0: the recursively updated residual) or per outer step
 * (refine = 1: the outer residual F - A u; where a provisional double-float
 * residual was recomputed in FP64, the FP64 value).  Writes min(*len,
 * max_len) values to host_out (may be NULL to ask for the length) and the
 * length to *len; 0 before the first solve.  Errors: STLS_EINVAL. */
int stls_residual_history(const stls_ctx *ctx, int b, double *host_out, int max_len, int *len);

/* Testing hook of the breakdown checks: replaces the eigenvalues of
 * direction `dir` (0..d-1 space, d time; n values in host memory) that the
 * FP64 preconditioner divides by (Algorithm 1, step 3), after the work queued
 * on the context's stream has finished.  With values that make some
 * lambda_t[i_t] + sum_k lambda_k[i_k] negative, P is indefinite and a solve
 * stops with STLS_EBREAKDOWN.  stls_get_factor(STLS_F_EIGVAL) returns the new
 * values; the eigenvectors are unchanged.  Errors: STLS_EINVAL for a mixed
 * precision context, dir out of range or NULL values. */
int stls_override_eigenvalues(stls_ctx *ctx, int dir, const double *lam_host);

/* Same as stls_get_factor but computed on the host from `prm` alone, without
 * a GPU or a context.  Returns STLS_EINVAL for invalid parameters, with the
 * reason in stls_last_error(NULL). */
int stls_host_factor(const stls_params *prm, int which, int dir, double *host_out);

/* Number of kernels this context has launched since creation. */
long long stls_launch_count(const stls_ctx *ctx);

/* Per-phase device timing of solves.  When enabled, stls_solve records CUDA
 * events around each phase; stls_phase_times returns, for phase ids
 * 0 = A x in FP64, 1 = P^{-1} r, 2 = CG vector updates and reductions,
 * 3 = A x in FP32 (refinement form), the summed milliseconds and the number
 * of executions since the last reset (arrays of 4).  Without timing, the
 * refinement form runs each inner flexible-CG loop as one launch of a CUDA
 * graph (a while node whose condition the last kernel of each step sets on
 * the device: no host round trip per step); with timing on, the host drives
 * the loop step by step so that the events can bracket each phase.  Both
 * run the same kernels in the same order, so results are identical. */
int stls_enable_timing(stls_ctx *ctx, int on);
int stls_phase_times(stls_ctx *ctx, double *ms_out4, long long *count_out4);
/* As stls_phase_times for the first min(n, 5) phase ids, adding
 * 4 = A x in double-float arithmetic (the refinement form's provisional
 * residuals, with the split of u).  ms_out, count_out: n entries or NULL. */
int stls_phase_times_n(stls_ctx *ctx, int n, double *ms_out, long long *count_out);

/* ---- local operations of a time-slab decomposition ----------------------------
 * The paper leaves parallel solvers to future work (Sec. 1 and 6); these calls
 * are the per-rank parts of a decomposition in which rank r owns the time
 * slices [t0_r, t1_r) of every right-hand side (vectors of B x (t1-t0) x N_s
 * entries, colexicographic within a slice).  A x (Eq. A_kron) is local in
 * space and banded in time: each rank forms the spatial factors of its slices,
 * exchanges p_t slices with each neighbour and applies the time band
 * (stls_slab_spatial, stls_slab_time).  Algorithm 1 is local in space and
 * dense in time: forward spatial products on the rank's slices, an
 * all-to-all that hands rank r a range [s0_r, s1_r) of spatial indices for
 * all times, the time products and the division on that range, the reverse
 * all-to-all and the backward spatial products (stls_fd_spatial,
 * stls_fd_time_chunk).  CG needs per-right-hand-side inner products, summed
 * over ranks, and vector updates (stls_vec_dot, stls_vec_axpby).  The
 * exchanges themselves belong to the caller (paper_1809_10026_gb300.timeslab).
 * All calls are FP64, need geometry = 0, and run on the context's stream. */

/* Spatial factors of Eq. A_kron on ns stacked spatial slices (any time slices
 * of any right-hand sides, 1 <= ns <= B n_t): Ms = M_s x, Js = J_s x,
 * Ls = L_s x per slice; any output may be NULL.  x, Ms, Js, Ls: device,
 * ns x N_s. */
int stls_slab_spatial(stls_ctx *ctx, const double *x, long long ns, double *Ms, double *Js, double *Ls);

/* Time rows [t0, t1) of y = (K_t x M_s + M_t x J_s + W_t x L_s) x from the
 * spatial factors of the slices [e0, e1) (the rank's rows and the halos):
 * Ms_ext, Js_ext: device, B x (e1-e0) x N_s; requires
 * 0 <= e0 <= t0 < t1 <= e1 <= n_t, e0 <= max(0, t0 - p_t) and
 * e1 >= min(n_t, t1 + p_t).  Ls_last: device, B x N_s, L_s x of the last time
 * slice, used (and then required) when t1 = n_t.  y: device,
 * B x (t1-t0) x N_s. */
int stls_slab_time(stls_ctx *ctx, const double *Ms_ext, const double *Js_ext, int e0, int e1, int t0, int t1,
                   const double *Ls_last, double *y);

/* Spatial mode products of Algorithm 1 on ns stacked spatial slices:
 * forward != 0: y = (U_d^T x ... x U_1^T) x (step 2 without the time mode);
 * forward == 0: y = (U_d x ... x U_1) x (step 4 without it).
 * x, y: device, ns x N_s, 1 <= ns <= B n_t, must not overlap. */
int stls_fd_spatial(stls_ctx *ctx, const double *x, double *y, long long ns, int forward);

/* The time part of Algorithm 1 on the spatial indices [s0, s1): y = U_t ((U_t^T x)
 * / (lambda_t[m] + lambda_s[s])), lambda_s[s] = sum_k lambda_k[i_k(s)] (steps 2-4 in
 * the time mode, with the division of step 3).  x, y: device, B x n_t x (s1-s0)
 * (the chunk's spatial index fastest), must not overlap; 0 <= s0 < s1 <= N_s. */
int stls_fd_time_chunk(stls_ctx *ctx, const double *x, double *y, long long s0, long long s1);

/* Per-right-hand-side inner products out_host[b] = sum_i x[b n + i] y[b n + i]
 * (b < B) in FP64, in a fixed order (deterministic); synchronizes the stream.
 * x, y: device, B x n. */
int stls_vec_dot(stls_ctx *ctx, const double *x, const double *y, long long n, double *out_host);

/* y[b n + i] = a_host[b] x[b n + i] + b_host[b] y[b n + i]: device vectors of
 * B x n, host arrays of B scalars. */
int stls_vec_axpby(stls_ctx *ctx, const double *a_host, const double *x, const double *b_host, double *y,
                   long long n);

/* ---- allocation-free preconditioner apply ------------------------------------
 * The paper has no counterpart to this entry point.  It serves callers that
 * cannot allocate device memory when they need the preconditioner: real-time
 * loops that cannot afford the allocator's latency or the device
 * synchronization that cudaMalloc and cudaFree can imply, and plugin hosts
 * that give a component a fixed memory budget and forbid it to allocate.
 * Such callers cannot create a context either (stls_create allocates), so
 * every input comes from the caller.
 *
 * Computes z = P^{-1} r in FP64 exactly as stls_apply_precond does in the
 * STLS_FP64 form (the same mode products and eigenvalue division), with the
 * two intermediate tensors held in a fixed 8 MiB device array inside the
 * library, which every GPU that loads the library keeps until process exit.
 *   d        spatial dimension 1..3
 *   n        host array of d+1 sizes: n_1..n_d, n_t (each 1..128)
 *   batch    right-hand sides; batch * prod(n) must not exceed 524288,
 *            otherwise STLS_EINVAL is returned and nothing is launched
 *   U        host array of d+1 DEVICE pointers to the eigenvector matrices
 *            U_1..U_d, U_t (row-major n_k x n_k, U^T M U = I), e.g. uploads of
 *            stls_host_factor(..., STLS_F_EIGVEC, k, ...)
 *   lam      host array of d+1 DEVICE pointers to the eigenvalues (length n_k)
 *   r, z     DEVICE, batch x N, colexicographic; r == z is allowed
 *   stream   cudaStream_t (NULL = legacy default stream)
 * Nothing is allocated or freed.  The first call on a device looks up the
 * array's device address with cudaGetSymbolAddress (with that device
 * current) and caches it with the device's context; make that first call
 * before any stream capture.  After cudaDeviceReset the next call looks the
 * address up again.  All calls share the array and nothing in it needs to
 * start at zero; calls whose kernels overlap on the GPU (different streams or
 * threads) race on it and must be serialized by the caller.  Errors:
 * STLS_EINVAL (sizes, NULL pointers), STLS_ECUDA (lookup or launch failure,
 * or a CUDA error already pending from earlier work, which is reported and
 * left set); text via stls_last_error(NULL). */
int stls_apply_precond_noalloc(int d, const int *n, int batch, const double *const *U,
                               const double *const *lam, const double *r, double *z,
                               void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* STLS_H */
