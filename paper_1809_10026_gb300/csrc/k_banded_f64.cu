// Banded mode products for the matrix-free system matrix (Eq. A_kron), in
// FP64 (the solver's residuals) or FP32 (the inner solves of the refinement
// form).
//
// One launch applies up to 12 terms out[t.out] += t.scale * (t.band x_k in[t.in])
// along one mode, where every band is a 1D Galerkin matrix of half-width p
// (Sec. 4.5: bands of width 2p+1).  One CTA owns 32 fibers of the mode-k
// unfolding; each input tile is staged in shared memory with p zero rows
// above and below, so the band never reads outside the tile.  A warp owns
// one row and 32 fibers, so the band coefficients are warp-uniform loads.
#include "kernels.h"

namespace stls {

namespace {

constexpr int kTC = 32;
constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;

template <typename T, int RPT>
__global__ void __launch_bounds__(kThreads)
    banded_kernel(BandSpecT<T> spec, ModeView v, long long ncols) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T *sm = reinterpret_cast<T *>(sm_raw);
  const int n = v.n, p = spec.p, w = 2 * p + 1;
  const int rows_pad = n + 2 * p;
  const int ntile = spec.n_in > spec.n_out ? spec.n_in : spec.n_out;
  const long long col0 = static_cast<long long>(blockIdx.x) * kTC;
  const int ncol_tile = static_cast<int>(min(static_cast<long long>(kTC), ncols - col0));
  const bool linear = v.inner == 1 && v.in_outer_stride == n;
  for (int t = 0; t < spec.n_in; ++t) {
    T *Xs = sm + static_cast<size_t>(t) * rows_pad * kTC;
    const T *src = spec.in[t];
    for (int e = threadIdx.x; e < p * kTC; e += kThreads) {
      Xs[e] = 0.0;
      Xs[(n + p) * kTC + e] = 0.0;
    }
    if (linear) {
      const T *s0 = src + col0 * n;
      for (int e = threadIdx.x; e < ncol_tile * n; e += kThreads) {
        int cc = e / n, j = e - cc * n;
        Xs[(j + p) * kTC + cc] = s0[e];
      }
      for (int e = threadIdx.x; e < n * kTC; e += kThreads) {
        int j = e / kTC, cc = e - j * kTC;
        if (cc >= ncol_tile) Xs[(j + p) * kTC + cc] = 0.0;
      }
    } else {
      for (int e = threadIdx.x; e < n * kTC; e += kThreads) {
        int j = e / kTC, cc = e - j * kTC;
        T val = T(0);
        if (cc < ncol_tile) {
          long long col = col0 + cc;
          long long o = col / v.inner, c = col - o * v.inner;
          val = src[o * v.in_outer_stride + static_cast<long long>(j) * v.inner + c];
        }
        Xs[(j + p) * kTC + cc] = val;
      }
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T acc[RPT][kMaxBandOut];
#pragma unroll
  for (int r = 0; r < RPT; ++r)
#pragma unroll
    for (int o = 0; o < kMaxBandOut; ++o) acc[r][o] = T(0);
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    const int i = warp + kWarps * r;
    if (i < n) {
      for (int t = 0; t < spec.n_terms; ++t) {
        const BandTermT<T> tm = spec.term[t];
        const T *Xs = sm + static_cast<size_t>(tm.in) * rows_pad * kTC + lane;
        const T *bnd = tm.band + static_cast<size_t>(i) * w;
        T s = T(0);
        for (int o = 0; o < w; ++o) s = fma(__ldg(bnd + o), Xs[(i + o) * kTC], s);
#pragma unroll
        for (int q = 0; q < kMaxBandOut; ++q)
          if (q == tm.out) acc[r][q] = fma(tm.scale, s, acc[r][q]);
      }
    }
  }
  __syncthreads();  // input tiles are reused for the outputs
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    const int i = warp + kWarps * r;
    if (i < n) {
#pragma unroll
      for (int q = 0; q < kMaxBandOut; ++q)
        if (q < spec.n_out) sm[static_cast<size_t>(q) * rows_pad * kTC + (i + p) * kTC + lane] = acc[r][q];
    }
  }
  __syncthreads();
  (void)ntile;
  const bool linear_out = v.inner == 1 && v.out_outer_stride == n && spec.last_add == nullptr;
  for (int q = 0; q < spec.n_out; ++q) {
    const T *Os = sm + static_cast<size_t>(q) * rows_pad * kTC;
    T *dst = spec.out[q];
    if (linear_out) {
      T *d0 = dst + col0 * n;
      for (int e = threadIdx.x; e < ncol_tile * n; e += kThreads) {
        int cc = e / n, i = e - cc * n;
        d0[e] = Os[(i + p) * kTC + cc];
      }
    } else {
      for (int e = threadIdx.x; e < n * kTC; e += kThreads) {
        int i = e / kTC, cc = e - i * kTC;
        if (cc >= ncol_tile) continue;
        long long col = col0 + cc;
        long long o = col / v.inner, c = col - o * v.inner;
        T val = Os[(i + p) * kTC + cc];
        if (spec.last_add != nullptr && q == spec.last_out && i == n - 1) val += spec.last_add[o * v.inner + c];
        dst[o * v.out_outer_stride + static_cast<long long>(i) * v.inner + c] = val;
      }
    }
  }
}

template <typename T, int RPT>
cudaError_t launch_rpt(const BandSpecT<T> &spec, const ModeView &v, cudaStream_t s) {
  const long long ncols = v.outer * v.inner;
  const int ntile = spec.n_in > spec.n_out ? spec.n_in : spec.n_out;
  const size_t smem = sizeof(T) * static_cast<size_t>(ntile) * (v.n + 2 * spec.p) * kTC;
  cudaError_t e = cudaFuncSetAttribute(banded_kernel<T, RPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  const long long grid = (ncols + kTC - 1) / kTC;
  if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  banded_kernel<T, RPT><<<static_cast<unsigned>(grid), kThreads, smem, s>>>(spec, v, ncols);
  return cudaGetLastError();
}

}  // namespace

template <typename T>
cudaError_t launch_banded(const BandSpecT<T> &spec, const ModeView &v, cudaStream_t s) {
  if (v.n < 1 || v.n > 128 || v.inner < 1 || v.outer < 0) return cudaErrorInvalidValue;
  if (spec.n_in < 1 || spec.n_in > kMaxBandIn || spec.n_out < 1 || spec.n_out > kMaxBandOut ||
      spec.n_terms < 1 || spec.n_terms > kMaxBandTerms || spec.p < 0)
    return cudaErrorInvalidValue;
  for (int t = 0; t < spec.n_terms; ++t)
    if (spec.term[t].in < 0 || spec.term[t].in >= spec.n_in || spec.term[t].out < 0 ||
        spec.term[t].out >= spec.n_out)
      return cudaErrorInvalidValue;
  if (v.outer == 0) return cudaSuccess;
  switch ((v.n + kWarps - 1) / kWarps) {
    case 1: return launch_rpt<T, 1>(spec, v, s);
    case 2: return launch_rpt<T, 2>(spec, v, s);
    case 3: return launch_rpt<T, 3>(spec, v, s);
    case 4: return launch_rpt<T, 4>(spec, v, s);
    case 5: return launch_rpt<T, 5>(spec, v, s);
    case 6: return launch_rpt<T, 6>(spec, v, s);
    case 7: return launch_rpt<T, 7>(spec, v, s);
    default: return launch_rpt<T, 8>(spec, v, s);
  }
}

template cudaError_t launch_banded<double>(const BandSpecT<double> &, const ModeView &, cudaStream_t);
template cudaError_t launch_banded<float>(const BandSpecT<float> &, const ModeView &, cudaStream_t);

}  // namespace stls
