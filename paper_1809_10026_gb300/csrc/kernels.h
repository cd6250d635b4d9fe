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

// ---- dense mode product: out = in x_k W (Algorithm 1, steps 2 and 4) -----------------
// out(o, i, c) = sum_j W[i * n + j] in(o, j, c).  If lam_row != nullptr the
// result is divided by lam_row[i] + lam_col[c] (Algorithm 1, step 3).
cudaError_t launch_modeprod_f64(const double *in, double *out, const double *W, const ModeView &v,
                                const double *lam_row, const double *lam_col, cudaStream_t s);

// ---- banded multi-term mode product (A x, Eq. A_kron) ----------------------------------
constexpr int kMaxBandIn = 4, kMaxBandOut = 4, kMaxBandTerms = 8;
struct BandTerm {
  const double *band;  // n x (2p+1) band storage of a 1D matrix
  int in, out;         // input and output slots
  double scale;
};
struct BandSpec {
  const double *in[kMaxBandIn];
  double *out[kMaxBandOut];
  int n_in, n_out, n_terms, p;
  BandTerm term[kMaxBandTerms];
  // optional: out[last_out](o, n-1, c) += last_add[o * inner + c]  (the W_t term)
  const double *last_add;
  int last_out;
};
cudaError_t launch_banded_f64(const BandSpec &spec, const ModeView &v, cudaStream_t s);

// ---- CG vector kernels with deterministic grid reductions --------------------------
struct CGState {
  double rz, pq, alpha, beta, rr, nF2, rel_res, true_rr;
  int active, iters, status, pad;
};
struct RedWork {
  double *partials;    // [batch][grid][2]
  unsigned *tickets;   // [batch], zero between kernels
  int grid;            // blocks per right-hand side
};
int red_grid_for(long long n);

cudaError_t launch_cg_init(const double *F, double *x, double *r, long long N, int B, CGState *st,
                           RedWork rw, cudaStream_t s);
cudaError_t launch_cg_alpha(const double *p, const double *q, long long N, int B, CGState *st,
                            RedWork rw, cudaStream_t s);
cudaError_t launch_cg_xr(double *x, double *r, const double *p, const double *q, long long N, int B,
                         double tol, CGState *st, RedWork rw, cudaStream_t s);
cudaError_t launch_cg_beta(const double *z, const double *r, const double *q, long long N, int B,
                           int flexible, int first, CGState *st, RedWork rw, cudaStream_t s);
cudaError_t launch_cg_p(const double *z, double *p, long long N, int B, int first, CGState *st,
                        cudaStream_t s);
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

}  // namespace stls
