// Dense FP64 mode products of the fast-diagonalization solve (Algorithm 1,
// steps 2 and 4): out = in x_k W with W = U_k^T (forward) or U_k (backward),
// n_k <= 128.  The eigenvalue division of step 3 is fused into the store of
// the forward time product.
//
// One CTA owns TC = 64 fibers (columns of the mode-k unfolding) and all n
// rows.  W (transposed) and the n x 64 tile live in shared memory; each of
// the 256 threads accumulates a ceil(n/16) x 4 register tile.  On GB300 the
// FP64 pipe (about 2 DFMA per clock per SM) bounds this kernel, not memory.
#include "kernels.h"

namespace stls {

namespace {

constexpr int kTC = 64;
constexpr int kThreads = 256;

template <int RPT>
__global__ void __launch_bounds__(kThreads)
    modeprod_f64_kernel(const double *__restrict__ in, double *__restrict__ out,
                        const double *__restrict__ W, ModeView v, long long ncols,
                        const double *__restrict__ lam_row, const double *__restrict__ lam_col) {
  extern __shared__ double sm[];
  const int n = v.n;
  double *Ws = sm;          // Ws[j * n + i] = W[i][j]
  double *Xs = sm + n * n;  // Xs[j * kTC + cc]
  const long long col0 = static_cast<long long>(blockIdx.x) * kTC;
  const int ncol_tile = static_cast<int>(min(static_cast<long long>(kTC), ncols - col0));
  for (int e = threadIdx.x; e < n * n; e += kThreads) {
    int i = e / n, j = e - i * n;
    Ws[j * n + i] = W[e];
  }
  const bool linear = v.inner == 1 && v.in_outer_stride == n;
  if (linear) {
    const double *src = in + col0 * n;
    for (int e = threadIdx.x; e < ncol_tile * n; e += kThreads) {
      int cc = e / n, j = e - cc * n;
      Xs[j * kTC + cc] = src[e];
    }
  } else {
    for (int e = threadIdx.x; e < n * kTC; e += kThreads) {
      int j = e / kTC, cc = e - j * kTC;
      double val = 0.0;
      if (cc < ncol_tile) {
        long long col = col0 + cc;
        long long o = col / v.inner, c = col - o * v.inner;
        val = in[o * v.in_outer_stride + static_cast<long long>(j) * v.inner + c];
      }
      Xs[e] = val;
    }
  }
  __syncthreads();
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[RPT][4];
#pragma unroll
  for (int r = 0; r < RPT; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[r][q] = 0.0;
  for (int j = 0; j < n; ++j) {
    double x[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) x[q] = Xs[j * kTC + tx + 16 * q];
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      int i = ty + 16 * r;
      double w = i < n ? Ws[j * n + i] : 0.0;
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[r][q] = fma(w, x[q], acc[r][q]);
    }
  }
  __syncthreads();  // Xs is reused as the output tile
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    int i = ty + 16 * r;
    if (i < n) {
#pragma unroll
      for (int q = 0; q < 4; ++q) Xs[i * kTC + tx + 16 * q] = acc[r][q];
    }
  }
  __syncthreads();
  const bool linear_out = v.inner == 1 && v.out_outer_stride == n && lam_row == nullptr;
  if (linear_out) {
    double *dst = out + col0 * n;
    for (int e = threadIdx.x; e < ncol_tile * n; e += kThreads) {
      int cc = e / n, i = e - cc * n;
      dst[e] = Xs[i * kTC + cc];
    }
  } else {
    for (int e = threadIdx.x; e < n * kTC; e += kThreads) {
      int i = e / kTC, cc = e - i * kTC;
      if (cc >= ncol_tile) continue;
      long long col = col0 + cc;
      long long o = col / v.inner, c = col - o * v.inner;
      double val = Xs[e];
      if (lam_row != nullptr) val = val / (lam_row[i] + lam_col[c]);
      out[o * v.out_outer_stride + static_cast<long long>(i) * v.inner + c] = val;
    }
  }
}

template <int RPT>
cudaError_t launch_rpt(const double *in, double *out, const double *W, const ModeView &v,
                       const double *lam_row, const double *lam_col, cudaStream_t s) {
  const long long ncols = v.outer * v.inner;
  const size_t smem = sizeof(double) * (static_cast<size_t>(v.n) * v.n + static_cast<size_t>(v.n) * kTC);
  cudaError_t e = cudaFuncSetAttribute(modeprod_f64_kernel<RPT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  const long long grid = (ncols + kTC - 1) / kTC;
  if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  modeprod_f64_kernel<RPT><<<static_cast<unsigned>(grid), kThreads, smem, s>>>(in, out, W, v, ncols,
                                                                               lam_row, lam_col);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_modeprod_f64(const double *in, double *out, const double *W, const ModeView &v,
                                const double *lam_row, const double *lam_col, cudaStream_t s) {
  if (v.n < 1 || v.n > 128 || v.inner < 1 || v.outer < 0) return cudaErrorInvalidValue;
  if (v.outer == 0) return cudaSuccess;
  switch ((v.n + 15) / 16) {
    case 1: return launch_rpt<1>(in, out, W, v, lam_row, lam_col, s);
    case 2: return launch_rpt<2>(in, out, W, v, lam_row, lam_col, s);
    case 3: return launch_rpt<3>(in, out, W, v, lam_row, lam_col, s);
    case 4: return launch_rpt<4>(in, out, W, v, lam_row, lam_col, s);
    case 5: return launch_rpt<5>(in, out, W, v, lam_row, lam_col, s);
    case 6: return launch_rpt<6>(in, out, W, v, lam_row, lam_col, s);
    case 7: return launch_rpt<7>(in, out, W, v, lam_row, lam_col, s);
    default: return launch_rpt<8>(in, out, W, v, lam_row, lam_col, s);
  }
}

}  // namespace stls
