// Tensor-core fast-diagonalization solve (Algorithm 1, steps 2-4) for the
// mixed-precision form, sm_103a (tcgen05 + bulk TMA copies).
//
// Each of the 2(d+1) mode products is one launch of a persistent kernel that
// computes, for tiles of 128 fibers of the mode-k unfolding,
//     D[f][m] = sum_k X[f][k] * W[m][k]          (W = U_k^T forward, U_k backward)
// with tcgen05.mma: A = the fiber tile (M = 128, K = n_k padded), B = W
// (N = n_k padded to 16, K-major), D = FP32 accumulators in tensor memory
// (TMEM lane = fiber, column = output index m).  Operands are BF16 (kind::f16)
// or TF32 (kind::tf32), in the canonical no-swizzle K-major shared-memory
// layout: 8-row x 16-byte core matrices, 8-row groups 128 B apart (SBO), and
// 16-byte K chunks LBO apart.
//
// Layout rotation.  The tensor is stored with one mode fastest; the pass for
// mode k reads it with mode k fastest, so a fiber is n_k contiguous entries
// and a tile of 128 fibers is one contiguous block, fetched by a single
// cp.async.bulk into shared memory (double-buffered, completion tracked by an
// mbarrier transaction count).  The pass writes its output with mode k
// slowest: entry (m, f) goes to m * (N / n_k) + f, which is the layout with
// mode k+1 fastest, and for each m a warp stores 32 consecutive fibers.  The
// first pass reads r in its natural order (mode 1 fastest); after 2(d+1)
// passes the order is natural again and the last pass writes z.
//
// The first pass reads FP64 r, the last writes FP64 z; the 2d intermediate
// tensors are BF16 (kind::f16) or FP32 (kind::tf32).  The division by the
// eigenvalue sum lambda_t[i_t] + sum_k lambda_k[i_k] (step 3) is fused into
// the epilogue of the forward time product, whose fibers are exactly the
// colexicographic spatial indices; it is done in FP32 from the FP64
// eigenvalues rounded once.
//
// Every wait on an mbarrier is bounded: on timeout the kernel records an
// error code in host-mapped memory, waits once more (bounded) for its own
// copies and MMAs, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>

#include "tc_fd.h"

namespace stls {

namespace {

constexpr int kFib = 128;      // fibers per tile = MMA M = TMEM lanes
constexpr int kThreads = 128;  // warp w owns TMEM lanes 32w .. 32w+31
constexpr uint32_t kTmemCols = 128;
constexpr uint32_t kSpinLimit = 1u << 24;
constexpr int kMaxBlocksPerSM = 4;  // 4 x 128 TMEM columns = 512 per SM
constexpr int kSmemPerSM = 227 * 1024;

enum { KIND_BF16 = 0, KIND_TF32 = 1 };

struct TcPass {
  const void *in;
  void *out;
  const uint8_t *bimg;  // canonical smem image of W (B operand)
  long long nfib;       // fibers in the batch = B * N / n
  long long fib_per_b;  // N / n
  long long N;          // entries per right-hand side
  int n, kp, np;        // mode size, padded K, padded N
  int bytes_raw;        // one raw input tile: 128 * n * sizeof(InT)
  int bytes_a, bytes_b; // A tile and B image in shared memory
  int bulk;             // 1: input 16-byte aligned, full tiles use bulk copies
  uint32_t idesc;
  uint32_t lbo_b;       // K-chunk stride of the B image
  const float *lam_t;   // division (forward time pass only)
  const float *lam_s;
  int *err;             // host-mapped error word
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr >> 4) & 0x3FFFu);
  d |= static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16;
  d |= static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32;
  d |= 1ull << 46;  // descriptor version for tcgen05; swizzle mode 0 = none
  return d;
}

__device__ __forceinline__ void mma_issue(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate, int kind) {
  if (kind == KIND_BF16) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
  } else {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
  }
}

__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity) {
  for (uint32_t it = 0; it < kSpinLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred P1;\nmbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n"
        "selp.b32 %0, 1, 0, P1;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// One bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned)
// from global to shared memory, completing a transaction on `mbar`.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint32_t mbar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(mbar)
      : "memory");
}

__device__ __forceinline__ float to_f32(double v) { return static_cast<float>(v); }
__device__ __forceinline__ float to_f32(float v) { return v; }
__device__ __forceinline__ float to_f32(__nv_bfloat16 v) { return __bfloat162float(v); }

__device__ __forceinline__ void store_out(double *p, float v) { *p = static_cast<double>(v); }
__device__ __forceinline__ void store_out(float *p, float v) { *p = v; }
__device__ __forceinline__ void store_out(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }

__device__ __forceinline__ uint32_t to_tf32(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return r;
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  uint32_t r;
  memcpy(&r, &h, 4);
  return r;
}

template <typename InT, typename OutT, int KIND, bool DIVIDE>
__global__ void __launch_bounds__(kThreads) tc_modeprod_kernel(TcPass a) {
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ uint32_t tmem_holder;
  __shared__ int flag_ok;
  __shared__ __align__(8) uint64_t mbar_mma;
  __shared__ __align__(8) uint64_t mbar_load[2];
  const int tid = threadIdx.x, warp = tid >> 5;
  uint8_t *sA = smem + 2 * a.bytes_raw;
  uint8_t *sB = sA + a.bytes_a;
  const uint32_t mma_bar = smem_u32(&mbar_mma);
  const uint32_t load_bar0 = smem_u32(&mbar_load[0]);  // stage s uses load_bar0 + 8 s
  const uint32_t raw0 = smem_u32(smem);                // stage s uses raw0 + s * bytes_raw
  const long long ntiles = (a.nfib + kFib - 1) / kFib;
  const long long nfull = a.bulk ? a.nfib / kFib : 0;  // tiles fetched by bulk copies
  const InT *in = static_cast<const InT *>(a.in);

  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mma_bar));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(load_bar0));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(load_bar0 + 8));
    asm volatile("fence.mbarrier_init.release.cluster;");
    asm volatile("fence.proxy.async.shared::cta;");
    flag_ok = 1;
    // prefetch this CTA's first two tiles
    for (int i = 0; i < 2; ++i) {
      const long long t = blockIdx.x + static_cast<long long>(i) * gridDim.x;
      if (t < nfull)
        bulk_load(raw0 + i * a.bytes_raw, in + t * kFib * a.n, static_cast<uint32_t>(a.bytes_raw),
                  load_bar0 + 8 * i);
    }
  }
  {
    const uint4 *src = reinterpret_cast<const uint4 *>(a.bimg);
    uint4 *dst = reinterpret_cast<uint4 *>(sB);
    for (int i = tid; i < a.bytes_b / 16; i += kThreads) dst[i] = src[i];
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_holder)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_holder;

  constexpr int esz = KIND == KIND_BF16 ? 2 : 4;
  constexpr int kcw = 16 / esz;                      // K values per 16-byte chunk
  constexpr int kstep = KIND == KIND_BF16 ? 16 : 8;  // K per MMA instruction
  const int nchunk = a.kp / kcw;
  const uint32_t lbo_a = (kFib / 8) * 128;  // 2048 B between K chunks of the A tile
  const uint32_t sA_addr = smem_u32(sA), sB_addr = smem_u32(sB);
  uint32_t mma_phase = 0;

  int i = 0;
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
    const int s = i & 1;
    const bool full = t < nfull;
    if (full) {
      if (!mbar_wait(load_bar0 + 8 * s, static_cast<uint32_t>((i >> 1) & 1))) flag_ok = 0;
    }
    __syncthreads();
    if (!flag_ok) break;
    const long long f = t * kFib + tid;
    const bool valid = f < a.nfib;
    const InT *src = full ? reinterpret_cast<const InT *>(smem + s * a.bytes_raw) + tid * a.n : in + f * a.n;
    // this fiber's K values -> 16-byte chunks of the canonical layout
    uint8_t *rowp = sA + (tid >> 3) * 128 + (tid & 7) * 16;
    for (int ch = 0; ch < nchunk; ++ch) {
      float v[8];
#pragma unroll
      for (int j = 0; j < kcw; ++j) {
        const int k = ch * kcw + j;
        v[j] = (valid && k < a.n) ? to_f32(src[k]) : 0.f;
      }
      uint4 pk;
      if (KIND == KIND_BF16) {
        pk.x = pack_bf16(v[0], v[1]);
        pk.y = pack_bf16(v[2], v[3]);
        pk.z = pack_bf16(v[4], v[5]);
        pk.w = pack_bf16(v[6], v[7]);
      } else {
        pk.x = to_tf32(v[0]);
        pk.y = to_tf32(v[1]);
        pk.z = to_tf32(v[2]);
        pk.w = to_tf32(v[3]);
      }
      *reinterpret_cast<uint4 *>(rowp + ch * lbo_a) = pk;
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (tid == 0) {
      // raw[s] is free again: fetch the tile two steps ahead
      const long long t2 = t + 2LL * gridDim.x;
      if (t2 < nfull)
        bulk_load(raw0 + s * a.bytes_raw, in + t2 * kFib * a.n, static_cast<uint32_t>(a.bytes_raw),
                  load_bar0 + 8 * s);
      asm volatile("tcgen05.fence::after_thread_sync;");
      const int nsteps = a.kp / kstep;
      for (int st = 0; st < nsteps; ++st) {
        // one instruction consumes two 16-byte K chunks
        const uint64_t ad = make_desc(sA_addr + 2 * st * lbo_a, lbo_a, 128);
        const uint64_t bd = make_desc(sB_addr + 2 * st * a.lbo_b, a.lbo_b, 128);
        mma_issue(tmem, ad, bd, a.idesc, st > 0 ? 1u : 0u, KIND);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       mma_bar)
                   : "memory");
      if (!mbar_wait(mma_bar, mma_phase)) {
        *reinterpret_cast<volatile int *>(a.err) = 1;
        mbar_wait(mma_bar, mma_phase);  // give in-flight MMAs one more bounded chance
        flag_ok = 0;
      }
    }
    mma_phase ^= 1u;
    __syncthreads();
    if (!flag_ok) break;
    asm volatile("tcgen05.fence::after_thread_sync;");
    // epilogue: TMEM lane = fiber (this thread), columns = output index m;
    // entry (m, fiber) goes to m * (N / n) + fiber within its right-hand side
    long long b = 0, fl = 0;
    if (valid) {
      b = f / a.fib_per_b;
      fl = f - b * a.fib_per_b;
    }
    OutT *dst = static_cast<OutT *>(a.out) + b * a.N + fl;
    const float lam_c = (DIVIDE && valid) ? a.lam_s[fl] : 0.f;
    for (int cb = 0; cb < a.np / 16; ++cb) {
      uint32_t r[16];
      const uint32_t taddr = tmem + (static_cast<uint32_t>(warp * 32) << 16) + cb * 16;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
          "[%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
            "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
            "=r"(r[14]), "=r"(r[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (valid) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int m = cb * 16 + j;
          if (m < a.n) {
            float val = __uint_as_float(r[j]);
            if (DIVIDE) val = val / (a.lam_t[m] + lam_c);
            store_out(dst + static_cast<long long>(m) * a.fib_per_b, val);
          }
        }
      }
    }
  }
  if (!flag_ok && tid == 0) {
    *reinterpret_cast<volatile int *>(a.err) = 1;
    // let this CTA's outstanding bulk copies land before its shared memory goes away
    for (int k = 0; k < 2; ++k) {
      const long long t = blockIdx.x + static_cast<long long>(i + k) * gridDim.x;
      if (t < nfull) mbar_wait(load_bar0 + 8 * ((i + k) & 1), static_cast<uint32_t>(((i + k) >> 1) & 1));
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
  }
}

// ---- host side ------------------------------------------------------------------------
struct Mode {
  int n, kp, np;
  uint8_t *bimg_fwd, *bimg_bwd;
  int bytes_a, bytes_b;
  uint32_t lbo_b;
};

struct Impl {
  Mode mode[4];
  void *inter[2];
  float *lam_t, *lam_s;
  int *err_host, *err_dev;
  int sms;
};

uint32_t make_idesc(int kind, int M, int N) {
  uint32_t d = 0;
  d |= 1u << 4;  // D format: F32
  const uint32_t fmt = kind == KIND_BF16 ? 1u : 2u;  // BF16 (kind::f16) or TF32 (kind::tf32)
  d |= fmt << 7;   // A format
  d |= fmt << 10;  // B format
  // bits 15/16 = 0: A and B K-major
  d |= static_cast<uint32_t>(N >> 3) << 17;
  d |= static_cast<uint32_t>(M >> 4) << 24;
  return d;
}

// Canonical no-swizzle K-major image of W (np x kp, rows m, K contiguous in 16-byte chunks).
std::vector<uint8_t> b_image(const std::vector<double> &W, int n, int np, int kp, int kind, bool transpose) {
  const int esz = kind == KIND_BF16 ? 2 : 4, kcw = 16 / esz;
  const uint32_t lbo = static_cast<uint32_t>(np / 8) * 128;
  std::vector<uint8_t> img(static_cast<size_t>(kp / kcw) * lbo, 0);
  for (int m = 0; m < n; ++m)
    for (int k = 0; k < n; ++k) {
      const double w = transpose ? W[k * n + m] : W[m * n + k];
      const size_t off = static_cast<size_t>(k / kcw) * lbo + (m / 8) * 128 + (m % 8) * 16 + (k % kcw) * esz;
      if (kind == KIND_BF16) {
        __nv_bfloat16 h = __float2bfloat16_rn(static_cast<float>(w));
        memcpy(&img[off], &h, 2);
      } else {
        float f = static_cast<float>(w);
        uint32_t bits;
        memcpy(&bits, &f, 4);
        // round to nearest TF32 (ties away), keep the top 19 bits
        bits = (bits + 0x1000u) & 0xFFFFE000u;
        memcpy(&img[off], &bits, 4);
      }
    }
  return img;
}

template <typename InT, typename OutT, int KIND, bool DIVIDE>
cudaError_t launch_pass(TcPass p, int sms, cudaStream_t s) {
  p.bytes_raw = kFib * p.n * static_cast<int>(sizeof(InT));
  p.bulk = (reinterpret_cast<uintptr_t>(p.in) % 16 == 0) ? 1 : 0;
  if (2 * static_cast<size_t>(p.bytes_raw) + p.bytes_a + p.bytes_b + 1024 > static_cast<size_t>(kSmemPerSM)) {
    p.bulk = 0;  // two raw stages do not fit: every tile is gathered with direct loads
  }
  if (!p.bulk) p.bytes_raw = 0;
  const size_t smem = 2 * static_cast<size_t>(p.bytes_raw) + p.bytes_a + p.bytes_b;
  auto kern = tc_modeprod_kernel<InT, OutT, KIND, DIVIDE>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  const long long ntiles = (p.nfib + kFib - 1) / kFib;
  // resident CTAs per SM from the shared-memory budget (1 KB reserved per CTA)
  int per_sm = static_cast<int>(kSmemPerSM / (smem + 1024 + 64));
  if (per_sm > kMaxBlocksPerSM) per_sm = kMaxBlocksPerSM;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  long long grid = static_cast<long long>(sms) * per_sm;
  if (grid > ntiles) grid = ntiles;
  if (grid < 1) return cudaSuccess;
  kern<<<static_cast<unsigned>(grid), kThreads, smem, s>>>(p);
  return cudaGetLastError();
}

template <typename T>
cudaError_t dev_alloc(TcFd &tc, T **p, size_t count) {
  void *v = nullptr;
  cudaError_t e = cudaMalloc(&v, count * sizeof(T) + 16);
  if (e != cudaSuccess) return e;
  tc.allocations.push_back(v);
  *p = static_cast<T *>(v);
  return cudaSuccess;
}

}  // namespace

cudaError_t tc_fd_create(TcFd &tc, int precision, int d, const int *n, int B,
                         const std::vector<std::vector<double>> &U, const std::vector<std::vector<double>> &lam,
                         const double *lam_t_dev, const double *lam_s_dev, std::string &err) {
  tc.precision = precision;
  tc.d = d;
  tc.B = B;
  tc.Ns = 1;
  for (int k = 0; k < d; ++k) tc.Ns *= n[k];
  tc.N = tc.Ns * n[d];
  for (int k = 0; k <= d; ++k) tc.n[k] = n[k];
  const int kind = precision == 2 ? KIND_BF16 : KIND_TF32;  // STLS_MIXED_BF16 = 2, STLS_MIXED_TF32 = 1
  Impl *im = new Impl();
  std::memset(im, 0, sizeof(Impl));
  tc.impl = im;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&im->sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  int major = 0, minor = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  if (major != 10 || minor != 3) {
    err = "the tensor-core preconditioner needs an sm_103 (GB300) device";
    return cudaSuccess;
  }
  if ((e = cudaHostAlloc(reinterpret_cast<void **>(&im->err_host), sizeof(int), cudaHostAllocMapped)) != cudaSuccess)
    return e;
  *im->err_host = 0;
  if ((e = cudaHostGetDevicePointer(reinterpret_cast<void **>(&im->err_dev), im->err_host, 0)) != cudaSuccess)
    return e;
  if (tc_fd_fused_eligible(precision, d, n)) {
    e = tc_fd_fused_create(tc.fused, tc.allocations, d, n, B, U, lam, im->err_dev, err);
    if (e == cudaSuccess && err.empty()) tc.launches_per_apply = tc_fd_fused_launches(tc.fused);
    return e;
  }
  if (tc_fd_rot_eligible(precision, d, n, B)) {
    std::string rerr;
    e = tc_fd_rot_create(tc.rot, tc.allocations, d, n, B, U, lam, im->err_dev, rerr);
    if (e == cudaSuccess && rerr.empty()) {
      tc.launches_per_apply = tc_fd_rot_launches(tc.rot);
      return e;
    }
    // a tensor map or pipeline the sizes do not allow: per-mode kernels below
    tc_fd_rot_destroy(tc.rot);
    tc.rot = nullptr;
    if (e != cudaSuccess && e != cudaErrorInvalidConfiguration) return e;
    cudaGetLastError();
  }
  for (int k = 0; k <= d; ++k) {
    Mode &m = im->mode[k];
    m.n = n[k];
    if (m.n > 128) {
      err = "tensor-core preconditioner supports 1D sizes up to 128";
      return cudaSuccess;
    }
    m.np = (m.n + 15) / 16 * 16;
    const int kstep = kind == KIND_BF16 ? 16 : 8;
    m.kp = (m.n + kstep - 1) / kstep * kstep;
    const int esz = kind == KIND_BF16 ? 2 : 4, kcw = 16 / esz;
    m.lbo_b = static_cast<uint32_t>(m.np / 8) * 128;
    const int nch = m.kp / kcw;
    m.bytes_b = nch * static_cast<int>(m.lbo_b);
    m.bytes_a = nch * (kFib / 8) * 128;
    std::vector<uint8_t> fwd = b_image(U[k], m.n, m.np, m.kp, kind, true);   // W = U^T
    std::vector<uint8_t> bwd = b_image(U[k], m.n, m.np, m.kp, kind, false);  // W = U
    if ((e = dev_alloc(tc, &m.bimg_fwd, fwd.size())) != cudaSuccess) return e;
    if ((e = dev_alloc(tc, &m.bimg_bwd, bwd.size())) != cudaSuccess) return e;
    if ((e = cudaMemcpy(m.bimg_fwd, fwd.data(), fwd.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
    if ((e = cudaMemcpy(m.bimg_bwd, bwd.data(), bwd.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
  }
  const size_t esz_inter = kind == KIND_BF16 ? 2 : 4;
  for (int i = 0; i < 2; ++i) {
    uint8_t *p = nullptr;
    if ((e = dev_alloc(tc, &p, esz_inter * static_cast<size_t>(B) * tc.N)) != cudaSuccess) return e;
    im->inter[i] = p;
  }
  // FP32 copies of the FP64 eigenvalues for the fused division
  std::vector<double> lt(n[d]), ls(tc.Ns);
  if ((e = cudaMemcpy(lt.data(), lam_t_dev, sizeof(double) * n[d], cudaMemcpyDeviceToHost)) != cudaSuccess) return e;
  if ((e = cudaMemcpy(ls.data(), lam_s_dev, sizeof(double) * tc.Ns, cudaMemcpyDeviceToHost)) != cudaSuccess) return e;
  std::vector<float> ltf(lt.begin(), lt.end()), lsf(ls.begin(), ls.end());
  if ((e = dev_alloc(tc, &im->lam_t, ltf.size())) != cudaSuccess) return e;
  if ((e = dev_alloc(tc, &im->lam_s, lsf.size())) != cudaSuccess) return e;
  if ((e = cudaMemcpy(im->lam_t, ltf.data(), 4 * ltf.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
  if ((e = cudaMemcpy(im->lam_s, lsf.data(), 4 * lsf.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
  tc.launches_per_apply = 2 * (d + 1);
  return cudaSuccess;
}

namespace {

// The 2(d+1) passes; IO is the type of r and z (double, or float for the inner
// solves of the refinement form).
template <typename IO>
cudaError_t apply_passes(TcFd &tc, const IO *r, IO *z, cudaStream_t s) {
  Impl *im = static_cast<Impl *>(tc.impl);
  if (im == nullptr) return cudaErrorNotReady;
  const int d = tc.d, nprod = 2 * (d + 1);
  const int kind = tc.precision == 2 ? KIND_BF16 : KIND_TF32;
  for (int st = 0; st < nprod; ++st) {
    const bool fwd = st <= d;
    const int k = fwd ? st : st - d - 1;
    const Mode &m = im->mode[k];
    TcPass p{};
    p.in = st == 0 ? static_cast<const void *>(r) : im->inter[(st - 1) % 2];
    p.out = st == nprod - 1 ? static_cast<void *>(z) : im->inter[st % 2];
    p.bimg = fwd ? m.bimg_fwd : m.bimg_bwd;
    p.N = tc.N;
    p.fib_per_b = tc.N / m.n;
    p.nfib = static_cast<long long>(tc.B) * p.fib_per_b;
    p.n = m.n;
    p.kp = m.kp;
    p.np = m.np;
    p.bytes_a = m.bytes_a;
    p.bytes_b = m.bytes_b;
    p.lbo_b = m.lbo_b;
    p.idesc = make_idesc(kind, kFib, m.np);
    p.lam_t = im->lam_t;
    p.lam_s = im->lam_s;
    p.err = im->err_dev;
    const bool divide = fwd && k == d;
    cudaError_t e;
    if (kind == KIND_BF16) {
      if (st == 0)
        e = launch_pass<IO, __nv_bfloat16, KIND_BF16, false>(p, im->sms, s);
      else if (st == nprod - 1)
        e = launch_pass<__nv_bfloat16, IO, KIND_BF16, false>(p, im->sms, s);
      else if (divide)
        e = launch_pass<__nv_bfloat16, __nv_bfloat16, KIND_BF16, true>(p, im->sms, s);
      else
        e = launch_pass<__nv_bfloat16, __nv_bfloat16, KIND_BF16, false>(p, im->sms, s);
    } else {
      if (st == 0)
        e = launch_pass<IO, float, KIND_TF32, false>(p, im->sms, s);
      else if (st == nprod - 1)
        e = launch_pass<float, IO, KIND_TF32, false>(p, im->sms, s);
      else if (divide)
        e = launch_pass<float, float, KIND_TF32, true>(p, im->sms, s);
      else
        e = launch_pass<float, float, KIND_TF32, false>(p, im->sms, s);
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace

cudaError_t tc_fd_apply(TcFd &tc, const double *r, double *z, cudaStream_t s) {
  if (tc.fused != nullptr) return tc_fd_fused_apply<double>(tc.fused, r, z, s);
  if (tc.rot != nullptr) return tc_fd_rot_apply<double>(tc.rot, r, z, s);
  return apply_passes<double>(tc, r, z, s);
}

cudaError_t tc_fd_apply_f32(TcFd &tc, const float *r, float *z, cudaStream_t s) {
  if (tc.fused != nullptr) return tc_fd_fused_apply<float>(tc.fused, r, z, s);
  if (tc.rot != nullptr) return tc_fd_rot_apply<float>(tc.rot, r, z, s);
  return apply_passes<float>(tc, r, z, s);
}

int tc_fd_error(const TcFd &tc) {
  const Impl *im = static_cast<const Impl *>(tc.impl);
  return im == nullptr || im->err_host == nullptr ? 0 : *im->err_host;
}

const int *tc_fd_error_flag(const TcFd &tc) {
  const Impl *im = static_cast<const Impl *>(tc.impl);
  return im == nullptr ? nullptr : im->err_dev;
}

int tc_fd_launch_count(const TcFd &tc) { return tc.launches_per_apply; }

float *tc_fd_padded_input(TcFd &tc, int *n0, int *np0) {
  return tc.rot != nullptr ? tc_fd_rot_padded_input(tc.rot, n0, np0) : nullptr;
}

cudaError_t tc_fd_apply_f32_padded(TcFd &tc, float *z, cudaStream_t s) {
  if (tc.rot == nullptr) return cudaErrorInvalidValue;
  return tc_fd_rot_apply_padded(tc.rot, z, s);
}

void tc_fd_destroy(TcFd &tc) {
  if (tc.fused != nullptr) tc_fd_fused_destroy(tc.fused);
  tc.fused = nullptr;
  if (tc.rot != nullptr) tc_fd_rot_destroy(tc.rot);
  tc.rot = nullptr;
  for (void *p : tc.allocations) cudaFree(p);
  tc.allocations.clear();
  Impl *im = static_cast<Impl *>(tc.impl);
  if (im != nullptr) {
    if (im->err_host) cudaFreeHost(im->err_host);
    delete im;
  }
  tc.impl = nullptr;
}

}  // namespace stls
