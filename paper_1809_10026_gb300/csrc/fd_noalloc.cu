// Allocation-free FP64 preconditioner apply (stls_apply_precond_noalloc).
//
// Some callers cannot allocate device memory at the point where they need the
// preconditioner: real-time loops that must not pay for the allocator's
// latency or the device synchronization cudaMalloc and cudaFree can imply,
// and hosts that hand a plugin a fixed memory budget and forbid it from
// allocating on its own.  They may not be able to create a solver context
// either, since stls_create allocates.  For them this file offers the FP64
// fast-diagonalization solve z = P^{-1} r with every input supplied by the
// caller and the two intermediate tensors kept in a file-scope device array
// instead of allocated memory.
//
// The array is a fixed 8 MiB (2 x 2^19 doubles) that every GPU which loads
// the library holds until the process exits.  One call handles at most
// 2^19 = 524,288 entries (batch x N); larger requests are rejected with
// STLS_EINVAL before anything is launched.  All calls share the array, and
// every intermediate entry is written before it is read within a call, so
// nothing in it needs to start at zero; two calls whose kernels overlap on
// the GPU (different streams, or different host threads) overwrite each
// other's intermediates and must be serialized by the caller.
//
// Host code cannot use the array's name as a device address (it denotes a
// host-side shadow symbol), so the first call on each device looks up the
// real address with cudaGetSymbolAddress while that device is current and
// caches it together with the device's current context.  That first call
// therefore must happen before any stream capture.  A later call that finds
// another context current on the device (after cudaDeviceReset, which
// reloads the module and may move the array) looks the address up again.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/stls.h"

namespace stls {
void set_thread_error(const std::string &msg);
}

namespace {

constexpr long long kNoAllocMaxElems = 1LL << 19;  // batch * N per call
constexpr int kMaxDevices = 64;
constexpr int kTC = 64;
constexpr int kThreads = 256;

static __device__ __align__(256) double g_noalloc_scratch[2 * kNoAllocMaxElems];

std::mutex g_mutex;
double *g_scratch_ptr[kMaxDevices] = {};
CUcontext g_scratch_ctx[kMaxDevices] = {};

// The driver's cuCtxGetCurrent through the runtime's entry-point query, so
// that the library does not link libcuda directly.
using CtxGetCurrentFn = CUresult (*)(CUcontext *);
CtxGetCurrentFn ctx_get_current() {
  static CtxGetCurrentFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<CtxGetCurrentFn>(p);
  }
  return fn;
}

// out(o, i, c) = sum_j W(i, j) in(o, j, c) with W(i, j) = U[j][i] when
// `transposed` (forward products, W = U^T) and U[i][j] otherwise.  When
// `lam` is non-null (forward time product) the result is divided by
// lam_t[i] + sum_k lam_k[i_k(c)], the eigenvalue sum of Algorithm 1 step 3,
// with the spatial index c decomposed on the fly.
template <int RPT>
__global__ void __launch_bounds__(kThreads)
    noalloc_modeprod_kernel(const double *__restrict__ in, double *__restrict__ out,
                            const double *__restrict__ U, int transposed, int n, long long inner,
                            long long ncols, const double *__restrict__ lam_t, int d,
                            const double *__restrict__ lam0, const double *__restrict__ lam1,
                            const double *__restrict__ lam2, int n0, int n1) {
  extern __shared__ double sm[];
  double *Ws = sm;          // Ws[j * n + i] = W(i, j)
  double *Xs = sm + n * n;  // Xs[j * kTC + cc], later the output tile
  const long long col0 = static_cast<long long>(blockIdx.x) * kTC;
  const int ncol_tile = static_cast<int>(min(static_cast<long long>(kTC), ncols - col0));
  for (int e = threadIdx.x; e < n * n; e += kThreads) {
    int a = e / n, b = e - a * n;  // U[a][b]
    if (transposed)
      Ws[a * n + b] = U[e];  // W(b, a) = U[a][b]
    else
      Ws[b * n + a] = U[e];  // W(a, b) = U[a][b]
  }
  for (int e = threadIdx.x; e < n * kTC; e += kThreads) {
    int j = e / kTC, cc = e - j * kTC;
    double v = 0.0;
    if (cc < ncol_tile) {
      long long col = col0 + cc;
      long long o = col / inner, c = col - o * inner;
      v = in[(o * n + j) * inner + c];
    }
    Xs[e] = v;
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
  __syncthreads();
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    int i = ty + 16 * r;
    if (i < n) {
#pragma unroll
      for (int q = 0; q < 4; ++q) Xs[i * kTC + tx + 16 * q] = acc[r][q];
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n * kTC; e += kThreads) {
    int i = e / kTC, cc = e - i * kTC;
    if (cc >= ncol_tile) continue;
    long long col = col0 + cc;
    long long o = col / inner, c = col - o * inner;
    double v = Xs[e];
    if (lam_t != nullptr) {
      long long rem = c;
      double ls = 0.0;
      if (d >= 1) { ls += lam0[rem % n0]; rem /= n0; }
      if (d >= 2) { ls += lam1[rem % n1]; rem /= n1; }
      if (d >= 3) ls += lam2[rem];
      v = v / (lam_t[i] + ls);
    }
    out[(o * n + i) * inner + c] = v;
  }
}

template <int RPT>
cudaError_t launch(const double *in, double *out, const double *U, int transposed, int n, long long inner,
                   long long ncols, const double *lam_t, int d, const double *const *lam, const int *nn,
                   cudaStream_t s) {
  const size_t smem = sizeof(double) * (static_cast<size_t>(n) * n + static_cast<size_t>(n) * kTC);
  cudaError_t e = cudaFuncSetAttribute(noalloc_modeprod_kernel<RPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  const long long grid = (ncols + kTC - 1) / kTC;
  noalloc_modeprod_kernel<RPT><<<static_cast<unsigned>(grid), kThreads, smem, s>>>(
      in, out, U, transposed, n, inner, ncols, lam_t, d, lam[0], d >= 2 ? lam[1] : nullptr,
      d >= 3 ? lam[2] : nullptr, nn[0], d >= 2 ? nn[1] : 1);
  return cudaGetLastError();
}

cudaError_t launch_any(const double *in, double *out, const double *U, int transposed, int n, long long inner,
                       long long ncols, const double *lam_t, int d, const double *const *lam, const int *nn,
                       cudaStream_t s) {
  switch ((n + 15) / 16) {
    case 1: return launch<1>(in, out, U, transposed, n, inner, ncols, lam_t, d, lam, nn, s);
    case 2: return launch<2>(in, out, U, transposed, n, inner, ncols, lam_t, d, lam, nn, s);
    case 3: return launch<3>(in, out, U, transposed, n, inner, ncols, lam_t, d, lam, nn, s);
    case 4: return launch<4>(in, out, U, transposed, n, inner, ncols, lam_t, d, lam, nn, s);
    case 5: return launch<5>(in, out, U, transposed, n, inner, ncols, lam_t, d, lam, nn, s);
    case 6: return launch<6>(in, out, U, transposed, n, inner, ncols, lam_t, d, lam, nn, s);
    case 7: return launch<7>(in, out, U, transposed, n, inner, ncols, lam_t, d, lam, nn, s);
    default: return launch<8>(in, out, U, transposed, n, inner, ncols, lam_t, d, lam, nn, s);
  }
}

// Device address of the scratch array on the current device, looked up once
// per device and context.
int scratch_for_current_device(double **out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    stls::set_thread_error("stls_apply_precond_noalloc: no usable current CUDA device");
    return STLS_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_mutex);
  CUcontext ctx = nullptr;
  if (g_scratch_ptr[dev] != nullptr) {
    // cheap check that the context the address belongs to is still current
    CtxGetCurrentFn get = ctx_get_current();
    if (get != nullptr && get(&ctx) == CUDA_SUCCESS && ctx != nullptr && ctx != g_scratch_ctx[dev])
      g_scratch_ptr[dev] = nullptr;
  }
  if (g_scratch_ptr[dev] == nullptr) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      stls::set_thread_error(std::string("stls_apply_precond_noalloc: cudaGetSymbolAddress failed: ") +
                             cudaGetErrorString(e));
      return STLS_ECUDA;
    }
    CtxGetCurrentFn get = ctx_get_current();
    ctx = nullptr;
    if (get != nullptr) get(&ctx);
    g_scratch_ptr[dev] = static_cast<double *>(p);
    g_scratch_ctx[dev] = ctx;
  }
  *out = g_scratch_ptr[dev];
  return STLS_OK;
}

}  // namespace

extern "C" int stls_apply_precond_noalloc(int d, const int *n, int batch, const double *const *U,
                                          const double *const *lam, const double *r, double *z,
                                          void *cuda_stream) {
  if (d < 1 || d > 3 || n == nullptr || U == nullptr || lam == nullptr || r == nullptr || z == nullptr ||
      batch < 1) {
    stls::set_thread_error("stls_apply_precond_noalloc: invalid argument");
    return STLS_EINVAL;
  }
  long long N = 1;
  for (int k = 0; k <= d; ++k) {
    if (n[k] < 1 || n[k] > 128 || U[k] == nullptr || lam[k] == nullptr) {
      stls::set_thread_error("stls_apply_precond_noalloc: 1D sizes must be in [1, 128] with non-NULL factors");
      return STLS_EINVAL;
    }
    N *= n[k];
  }
  if (static_cast<long long>(batch) * N > kNoAllocMaxElems) {
    stls::set_thread_error("stls_apply_precond_noalloc: batch * N = " + std::to_string(batch * N) +
                           " exceeds the fixed scratch capacity of 524288 entries");
    return STLS_EINVAL;
  }
  double *scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc != STLS_OK) return rc;
  // An error left pending by earlier work would be read back after our first
  // launch and reported as ours: report it as what it is, and leave it set.
  const cudaError_t pending = cudaPeekAtLastError();
  if (pending != cudaSuccess) {
    stls::set_thread_error(std::string("stls_apply_precond_noalloc: an earlier CUDA error is pending: ") +
                           cudaGetErrorString(pending));
    return STLS_ECUDA;
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  double *tmp[2] = {scratch, scratch + kNoAllocMaxElems};
  const int nprod = 2 * (d + 1);
  const double *src = r;
  for (int st = 0; st < nprod; ++st) {
    const bool fwd = st <= d;
    const int k = fwd ? st : st - d - 1;
    long long inner = 1;
    for (int l = 0; l < k; ++l) inner *= n[l];
    const long long ncols = static_cast<long long>(batch) * N / n[k];
    double *dst = st == nprod - 1 ? z : tmp[st % 2];
    const bool divide = fwd && k == d;
    cudaError_t e = launch_any(src, dst, U[k], fwd ? 1 : 0, n[k], inner, ncols, divide ? lam[d] : nullptr, d,
                               lam, n, s);
    if (e != cudaSuccess) {
      stls::set_thread_error(std::string("stls_apply_precond_noalloc: launch failed: ") + cudaGetErrorString(e));
      return STLS_ECUDA;
    }
    src = dst;
  }
  return STLS_OK;
}
