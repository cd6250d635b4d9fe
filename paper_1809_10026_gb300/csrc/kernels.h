// Launch interfaces of the CUDA kernels (all FP64 unless stated).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/stls.h"

namespace stls {

// A tensor seen along one mode: (outer, n, inner), inner fastest.  Entry
// (o, i, c) of the input lives at base + o * in_outer_stride + i * inner + c.
struct ModeView {
  int n;                    // size of the contracted mode
  long long inner;          // product of the sizes of the faster modes
  long long outer;          // number of (n x inner) slabs
  long long in_outer_stride;
  long long out_outer_stride;
};

// Double-float number: the unevaluated sum h + l of two FP32 values with
// |l| <= ulp(h) / 2 (Dekker 1971), about 48 significant bits.  Products and
// sums of such pairs run on the FP32 pipe, 64 times the FP64 rate on GB300.
struct CGState;

struct alignas(8) dfloat {
  float h, l;
  dfloat() = default;
  __host__ __device__ constexpr explicit dfloat(float v) : h(v), l(0.f) {}
};

// ---- fused A x for two and three spatial directions (k_apply_a.cu) -------------------
// Band rows are padded to band_row_stride(p, sizeof(T)) elements (whole 16-byte
// vectors); b2K holds 2 K exactly.
constexpr int kFusedMaxP = 6;
int band_row_stride(int p, int elem_bytes);
bool fused_A_supported(int d, int p_s, int p_t);

template <typename T>
struct SliceArgs {
  const T *x;
  T *out_m, *out_j, *out_k;  // states after directions 1, 2 (out_k unused when ls_last is set)
  T *ls_last;                // two spatial directions: L_s x of the last time slice, per b
  const T *bM1, *bJ1, *bK1, *bM2, *bJ2, *bK2, *b2K2;
  long long slices;  // number of n2 x n1 slices
  long long out_area;  // elements from one slice of out_m, out_j, out_k to the next (>= n1 n2)
  int n1, n2, n_t, row_stride;
  int lo2, hi2;      // rows [lo2, hi2) of the direction-2 bands are all equal (uniform knots)
};
template <typename T>
struct ZArgs {
  const T *m, *j, *k;
  T *Ms, *Js, *ls_last;
  const T *bM, *bJ, *bK, *b2K;
  long long outer, inner;  // outer = B n_t, inner = n1 n2
  int n, n_t, row_stride;
  int lo, hi;              // rows [lo, hi) of the bands are all equal
};
// The CG step length fused into the last kernel of an FP32 A x: (p, y) per
// right-hand side with the same compensated accumulation and deterministic
// order as launch_cg_alpha, then alpha = rz / (p, y) with its checks.
struct AlphaFuse {
  const float *p;      // NULL: not fused
  CGState *st;
  double *partials;    // B * alpha_blocks(N_s) entries
  unsigned *tickets;   // B entries, zero between launches
};
int alpha_blocks(long long Ns);

template <typename T>
struct TArgs {
  const T *Ms, *Js, *ls_last;
  T *y;
  AlphaFuse fuse;  // FP32 only
  const T *bK, *bM;
  long long outer, inner;  // outer = B, inner = N_s
  int n, row_stride;
  int lo, hi;              // rows [lo, hi) of the bands are all equal
};
template <typename T>
struct FusedA {
  int d, p_s, p_t, n[3], n_t, B;
  const T *bM[3], *bJ[3], *bK[3], *b2K[3];  // padded spatial bands
  const T *bKt, *bMt;                       // padded time bands
  T *work[5];                               // d = 3: m, j', k, M_s x, J_s x; d = 2: work[3..4]
  T *ls_last;                               // B * N_s
  AlphaFuse fuse;                           // FP32: (p, A p) and alpha in the time kernel
  // rows [lo, hi) of every band of a direction are identical (the interior
  // rows of uniform-knot Galerkin matrices); lo = hi = 0 when none are
  int lo[3], hi[3], lo_t, hi_t;
  T iKt[2 * kFusedMaxP + 1], iMt[2 * kFusedMaxP + 1];  // host copy of the interior time band rows
  T i3[4][2 * kFusedMaxP + 1];  // host copy of the interior rows of M, J, 2K, K of direction 3
};
// Largest run of rows around the middle row of an n x stride band array in
// which every one of the given arrays has rows identical (bitwise) to its
// middle row; writes [lo, hi).
template <typename T>
void toeplitz_rows(const T *const *bands, int nbands, int n, int stride, int *lo, int *hi);
// y = A x; 2 launches (d = 2) or 3 (d = 3).  x, y: B * N values, colexicographic.
// T = double, float or dfloat (double-float arithmetic with FP32 operations).
template <typename T>
cudaError_t launch_fused_A(const FusedA<T> &f, const T *x, T *y, cudaStream_t s);
// Double-float images of B vectors of N FP64 values and back: y = x * 2^-k_b
// split into h + l, and x = 2^k_b (h + l) rounded to FP64, with k_b = 0 when
// `scale` is NULL, else the exponent of ||F_b|| (frexp of sqrt(scale[b].nF2)),
// so that the FP32 parts of a solution u stay far from FP32 overflow and
// underflow.
cudaError_t launch_df_split(const double *x, dfloat *y, long long N, int B, const CGState *scale,
                            cudaStream_t s);
cudaError_t launch_df_join(const dfloat *y, double *x, long long N, int B, const CGState *scale,
                           cudaStream_t s);

// ---- dense mode product: out = in x_k W (Algorithm 1, steps 2 and 4) -----------------
// out(o, i, c) = sum_j W[i * n + j] in(o, j, c).  If lam_row != nullptr the
// result is divided by lam_row[i] + lam_col[c] (Algorithm 1, step 3).
cudaError_t launch_modeprod_f64(const double *in, double *out, const double *W, const ModeView &v,
                                const double *lam_row, const double *lam_col, cudaStream_t s);

// ---- banded multi-term mode product (A x, Eq. A_kron), T = double or float --------
constexpr int kMaxBandIn = 4, kMaxBandOut = 4, kMaxBandTerms = 12;
template <typename T>
struct BandTermT {
  const T *band;  // n x (2p+1) band storage of a 1D matrix
  int in, out;    // input and output slots
  T scale;
};
template <typename T>
struct BandSpecT {
  const T *in[kMaxBandIn];
  T *out[kMaxBandOut];
  int n_in, n_out, n_terms, p;
  BandTermT<T> term[kMaxBandTerms];
  // optional: out[last_out](o, n-1, c) += last_add[o * inner + c]  (the W_t term)
  const T *last_add;
  int last_out;
};
using BandTerm = BandTermT<double>;
using BandSpec = BandSpecT<double>;
template <typename T>
cudaError_t launch_banded(const BandSpecT<T> &spec, const ModeView &v, cudaStream_t s);

inline cudaError_t launch_banded_f64(const BandSpec &spec, const ModeView &v, cudaStream_t s) {
  return launch_banded<double>(spec, v, s);
}

// ---- CG vector kernels with deterministic grid reductions --------------------------
struct CGState {
  double rz, pq, alpha, beta, rr, nF2, rel_res, true_rr;
  int active, iters, status, df_iters;  // df_iters: provisional double-float residuals
  int xpend;  // deferred x update: alpha p of the last x, r update is still owed to x
  int limit;      // inner solves: iteration cap of this outer step (graph loop condition)
  double tol_in;  // inner solves: relative-residual target (kernels given tol < 0 read it)
};
struct RedWork {
  double *partials;    // [batch][grid][2]
  unsigned *tickets;   // [batch], zero between kernels
  int grid;            // blocks per right-hand side
};
int red_grid_for(long long n);

cudaError_t launch_cg_init(const double *F, double *x, double *r, long long N, int B, CGState *st,
                           RedWork rw, cudaStream_t s);
// CG vector kernels for T = double (the solver) or float (inner solves of the
// refinement form); FP64 inner products accumulate in FP64, FP32 ones in
// compensated FP32 (twice-working-precision accuracy) per thread and FP64 across.
template <typename T>
cudaError_t launch_cg_alpha(const T *p, const T *q, long long N, int B, CGState *st, RedWork rw, cudaStream_t s);
template <typename T>
cudaError_t launch_cg_xr(T *x, T *r, const T *p, const T *q, long long N, int B, double tol, CGState *st,
                         RedWork rw, cudaStream_t s);
// cg_xr in FP32 that also writes r rounded to TF32 into rows of n0 values
// np0 apart (per right-hand side: N / n0 rows), the TF32 preconditioner's input.
// defer != 0: x is not updated here (see launch_cg_p and launch_ir_correct).
cudaError_t launch_cg_xr_pad(float *x, float *r, const float *p, const float *q, long long N, int B, double tol,
                             CGState *st, RedWork rw, float *rpad, int n0, int np0, int defer, cudaStream_t s);
// first < 0 (launch_cg_beta, launch_cg_p): the first step of the CG loop is
// the one with st.iters == 0, read on the device (a captured loop body).
template <typename T>
cudaError_t launch_cg_beta(const T *z, const T *r, const T *q, long long N, int B, int flexible, int first,
                           CGState *st, RedWork rw, cudaStream_t s);
// With x != NULL (FP32 inner solves after launch_cg_xr_pad with defer): also
// the deferred x += alpha p with the old p; `tickets` (zero between kernels)
// lets the last block clear the owed-update flag.
template <typename T>
cudaError_t launch_cg_p(const T *z, T *p, long long N, int B, int first, CGState *st, cudaStream_t s,
                        T *x = nullptr, unsigned *tickets = nullptr);
// Refinement form: FP32 inner right-hand side r64 2^-k (||r64|| = f 2^k,
// f in [0.5, 1)), FP64 correction of u, FP64 residual F - A u with the outer
// convergence test.
// (rpad != NULL: also r32 rounded to TF32 into rows of n0 values np0 apart,
// as launch_cg_xr_pad writes them.)
// The inner states also get tol_in = eta and limit = the iteration cap.
cudaError_t launch_ir_start(const double *r64, float *r32, float *d, long long N, int B, const CGState *outer,
                            CGState *inner, RedWork rw, float *rpad, int n0, int np0, double eta, int limit,
                            cudaStream_t s);
// One thread: sets the while-loop condition of a graph to "some right-hand
// side is active with iters < limit, and no tensor-core wait has failed"
// (err: the host-mapped failure flag of the preconditioner, or NULL).
cudaError_t launch_inner_cond(const CGState *st, int B, const int *err, cudaGraphConditionalHandle h,
                              cudaStream_t s);
// u += 2^k d (k: exponent of ||r64||, as ir_start scaled); with p != NULL, d
// first takes the x += alpha p that launch_cg_xr_pad deferred (inner[b].xpend,
// inner[b].alpha: one FP32 FMA per entry, as the CG update would have done); with udf != NULL
// also writes launch_df_split's image of the new u (scale from outer).
cudaError_t launch_ir_correct(double *u, const float *d, const float *p, const CGState *inner, dfloat *udf,
                              long long N, int B, const CGState *outer, cudaStream_t s);
// `count` = 1 when the residual ends an outer step, 0 when it re-evaluates the
// last one in FP64.
cudaError_t launch_ir_residual(const double *F, const double *Au, double *r64, long long N, int B, double tol,
                               int count, CGState *outer, RedWork rw, cudaStream_t s);
// Same with A u given as the double-float image 2^-k_b A u (launch_df_split's
// scale taken from `outer`).  The result is provisional: it updates the
// residual, its norm and the outer step count but never ends a solve or flags
// a non-finite value; the host confirms convergence (or a non-finite norm)
// with the FP64 residual.
cudaError_t launch_ir_residual_df(const double *F, const dfloat *Au, double *r64, long long N, int B,
                                  CGState *outer, RedWork rw, cudaStream_t s);
cudaError_t launch_true_residual(const double *F, const double *Ax, long long N, int B, CGState *st,
                                 RedWork rw, cudaStream_t s);

// ---- lifting helpers (Sec. 3.1) ----------------------------------------------------
// y(b, t, c) = e[t] * Ls(b, c) + m[t] * Js(b, c)
cudaError_t launch_lift_combine(const double *Ls, const double *Js, const double *e, const double *m,
                                double *y, long long Ns, int nt, int B, cudaStream_t s);
// a(b, c) = sum_t e[t] * lam(b, t, c), bsum(b, c) = sum_t m[t] * lam(b, t, c),
// gsum(b, c) = sum_t g(b, t, c)
cudaError_t launch_lift_reduce(const double *lam, const double *g, const double *e, const double *m,
                               double *a, double *bsum, double *gsum, long long Ns, int nt, int B,
                               cudaStream_t s);
// out = x + alpha * y (elementwise, n entries)
cudaError_t launch_axpy(const double *x, const double *y, double alpha, double *out, long long n,
                        cudaStream_t s);
// out[b] = sum_i x[b n + i] y[b n + i] (fixed order), B vectors of n entries
cudaError_t launch_vec_dot(const double *x, const double *y, long long n, int B, double *out, RedWork rw,
                           cudaStream_t s);
// y[b n + i] = ab[b] x[b n + i] + ab[B + b] y[b n + i]  (ab: device, 2B scalars)
cudaError_t launch_vec_axpby(const double *ab, const double *x, double *y, long long n, int B, cudaStream_t s);
// y[b, i] = x[b, i] * w[i] for B vectors of N entries (x == y allowed)
cudaError_t launch_scale(const double *x, const double *w, double *y, long long N, int B, cudaStream_t s);

}  // namespace stls
