// Tensor-core fast-diagonalization solve for the TF32 form (Algorithm 1,
// steps 2-4) on sm_103a: 2(d+1) rotation passes, one mode product each.
//
// Layout rotation.  Pass k reads the tensor with mode k fastest: fiber f (all
// other modes, mode k+1 fastest) holds n_k values, stored as a row of
// np_k = ceil4(n_k) FP32 values, so rows are 16-byte aligned and a tile of 128
// fibers is one 2D TMA box per 32 values of K (128-byte rows, 128-byte
// swizzle, values past n_k zero-filled by the TMA unit).  That box layout is
// the canonical K-major SW128 operand of tcgen05.mma kind::tf32 (8-row x
// 128-byte atoms, 1024 bytes apart), so the tile needs no conversion in
// shared memory: A = 128 fibers x K, B = the eigenvector matrix (N = n_k padded
// to 16 rows, K-major SW128 image built on the host), D = FP32 in tensor
// memory (lane = fiber, column = output index m).  A last partial group of at
// most 16 values of K (n_k = 65: one value) is not fetched as a whole 128-byte
// swizzled box but as boxes of 4 values (16-byte rows, no swizzle), which are
// the 8-row x 16-byte core matrices of the no-swizzle K-major layout (8-row
// groups 128 bytes apart, 4-value K chunks 2048 bytes apart): smaller stages,
// and on the 18.1M-unknown cube 343 instead of 346 us per apply.  The epilogue writes entry
// (m, f) as element i_{k+1} of fiber g + G m of the next pass (f = i_{k+1} +
// n_{k+1} g), i.e. with mode k slowest and mode k+1 fastest; after 2(d+1)
// passes the order is natural again.  For a fixed m a warp stores 32
// consecutive fibers, consecutive addresses.
//
// Rounding.  Every stored intermediate is rounded to TF32 (round to nearest,
// ties away: cvt.rna), so the MMA, which reads the top 19 bits of each FP32
// operand, uses it exactly; the first pass reads r in the same padded,
// rounded rows, written either by a padding kernel or directly by the
// producer of r (tc_fd_rot_padded_input: the inner CG updates of the
// refinement form), and the last pass writes z unrounded.  The
// division by lambda_t[m] + lambda_s[c] (step 3) is fused into the epilogue of
// the forward time pass, whose fibers are the colexicographic spatial indices
// c; FP32 (__fdividef), from the FP64 eigenvalues rounded once.
//
// Roles (one CTA per SM, persistent over tiles): warp 0 issues the TMA loads
// into a ring of shared-memory stages, warp 1 issues the MMAs into four
// tensor-memory accumulators in turn, and four groups of four warps drain one
// accumulator each (warp w reads TMEM lanes 32 (w mod 4) ..), so that four
// tiles' epilogues run at once.  Stages and accumulators are handed over by
// mbarriers; every wait is bounded, and on a timeout the kernel records the
// error, lets its own copies and MMAs finish (bounded), frees its tensor
// memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "tc_fd.h"
#include "tc_ptx.cuh"

namespace stls {

namespace {

constexpr int kAcc = 4;                   // tensor-memory accumulators, one epilogue group each
constexpr int kRotThreads = 64 + 128 * kAcc;  // warp 0 TMA, warp 1 MMA, 4 epilogue warps per accumulator
constexpr int kFib = 128;                 // fibers per tile = MMA M = TMEM lanes
constexpr int kBoxK = 32;                 // FP32 values per 128-byte swizzled row
constexpr uint32_t kBoxBytes = kFib * 128;
constexpr uint32_t kAccCols = 128;  // TMEM columns per accumulator (N <= 128)
constexpr int kMaxStages = 4;
constexpr int kSmemLimit = 227 * 1024;
constexpr int kStaticSmem = 1024;  // barriers, holder, eigenvalue copy

constexpr uint32_t kTailBoxBytes = kFib * 16;  // one 4-value box of the no-swizzle tail
constexpr int kTailMax = 16;                    // largest K tail fetched in 4-value boxes

struct RotArgs {
  void *out;
  const uint8_t *bimg;  // K-major SW128 image of W: nkb atoms of np rows x 128 bytes
  const float *lam_t, *lam_s;
  int *err;
  long long rows;       // fibers over the batch
  long long fib_per_b;  // fibers per right-hand side
  long long G;          // fib_per_b / n_next
  long long blk_out;    // output elements per right-hand side
  int n, nkb, ksteps, np, n_next, np_next, stages, round_out;
  int full_atoms;  // 32-value K groups fetched as SW128 boxes
  int tail_boxes;  // 4-value boxes of the no-swizzle tail (even; 0: none)
  uint32_t bytes_b, off_stage, idesc, stage_bytes;
};

__device__ __forceinline__ uint8_t *align1024(uint8_t *p) {
  return reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(p) + 1023) & ~static_cast<uintptr_t>(1023));
}

__device__ __forceinline__ void store_val(float *p, float v) { *p = v; }
__device__ __forceinline__ void store_val(double *p, float v) { *p = ptx::f32_to_f64(v); }

template <typename OutT, bool DIVIDE>
__global__ void __launch_bounds__(kRotThreads, 1) rot_kernel(const __grid_constant__ CUtensorMap tin,
                                                             const __grid_constant__ CUtensorMap ttail, RotArgs a) {
  extern __shared__ uint8_t smem_dyn[];
  __shared__ __align__(8) uint64_t bar_full[kMaxStages], bar_empty[kMaxStages], bar_tfull[kAcc], bar_tempty[kAcc];
  __shared__ uint32_t tmem_holder;
  __shared__ volatile int ok;
  __shared__ float s_lam_t[128];
  uint8_t *sm = align1024(smem_dyn);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int S = a.stages;
  const uint32_t stage_bytes = a.stage_bytes;
  const uint32_t sB = ptx::smem_u32(sm), st0 = ptx::smem_u32(sm + a.off_stage);
  const uint32_t full0 = ptx::smem_u32(&bar_full[0]), empty0 = ptx::smem_u32(&bar_empty[0]);
  const uint32_t tfull0 = ptx::smem_u32(&bar_tfull[0]), tempty0 = ptx::smem_u32(&bar_tempty[0]);
  const long long ntiles = (a.rows + kFib - 1) / kFib;

  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      ptx::mbar_init(full0 + 8 * s, 1);
      ptx::mbar_init(empty0 + 8 * s, 1);
    }
    for (int c = 0; c < kAcc; ++c) {
      ptx::mbar_init(tfull0 + 8 * c, 1);
      ptx::mbar_init(tempty0 + 8 * c, 4);  // one arrival per warp of the accumulator's group
    }
    ptx::mbar_init_fence();
    ok = 1;
  }
  {
    const uint4 *src = reinterpret_cast<const uint4 *>(a.bimg);
    for (uint32_t i = tid; i < a.bytes_b / 16; i += kRotThreads) reinterpret_cast<uint4 *>(sm)[i] = src[i];
    if (DIVIDE)
      for (int i = tid; i < 128; i += kRotThreads) s_lam_t[i] = i < a.n ? a.lam_t[i] : 0.f;
  }
  if (warp == 0) ptx::tmem_alloc(ptx::smem_u32(&tmem_holder), kAcc * kAccCols);
  ptx::fence_proxy_async();
  ptx::fence_before_sync();
  __syncthreads();
  ptx::fence_after_sync();
  const uint32_t tmem = tmem_holder;
  // Programmatic dependent launch: the next pass may start its prologue on the
  // SMs this grid leaves; this grid reads its input and overwrites the buffer
  // the previous pass read only once that pass has completed.
  asm volatile("griddepcontrol.launch_dependents;");
  asm volatile("griddepcontrol.wait;" ::: "memory");

  long long issued = 0, mmas = 0;  // warp 0 / warp 1, lane 0: for the error path
  if (warp == 0) {
    if (lane == 0) {
      long long i = 0;
      for (long long t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
        const int s = static_cast<int>(i % S);
        const uint32_t ph = static_cast<uint32_t>((i / S) & 1);
        if (!ptx::mbar_wait(empty0 + 8 * s, ph ^ 1u)) {
          ok = 0;
          break;
        }
        if (!ok) break;
        const uint32_t dst = st0 + s * stage_bytes;
        ptx::mbar_expect_tx(full0 + 8 * s, stage_bytes);
        for (int j = 0; j < a.full_atoms; ++j)
          ptx::tma_load_2d(dst + j * kBoxBytes, &tin, j * kBoxK, static_cast<int>(t * kFib), full0 + 8 * s);
        for (int j = 0; j < a.tail_boxes; ++j)  // x = 32 full_atoms + 4 j: 16-byte aligned
          ptx::tma_load_2d(dst + a.full_atoms * kBoxBytes + j * kTailBoxBytes, &ttail, a.full_atoms * kBoxK + 4 * j,
                           static_cast<int>(t * kFib), full0 + 8 * s);
        issued = i + 1;
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      long long i = 0;
      const uint32_t atom_b = static_cast<uint32_t>(a.np) * 128;
      for (long long t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
        const int s = static_cast<int>(i % S);
        const uint32_t ph = static_cast<uint32_t>((i / S) & 1);
        const int acc = static_cast<int>(i % kAcc);
        const uint32_t aph = static_cast<uint32_t>((i / kAcc) & 1);
        if (!ptx::mbar_wait(full0 + 8 * s, ph) || !ptx::mbar_wait(tempty0 + 8 * acc, aph ^ 1u)) {
          ok = 0;
          break;
        }
        if (!ok) break;
        ptx::fence_after_sync();
        const uint32_t A = st0 + s * stage_bytes, D = tmem + acc * kAccCols;
        const int kfull = 4 * a.full_atoms;
        for (int kk = 0; kk < a.ksteps; ++kk) {
          const int j = kk >> 2, w = kk & 3;  // 128-byte atom, 32-byte K step inside it
          const uint64_t ad = kk < kfull ? ptx::make_desc(A + j * kBoxBytes + w * 32, 16, 1024, 2)
                                         : ptx::make_desc(A + a.full_atoms * kBoxBytes + (kk - kfull) * 2 * kTailBoxBytes,
                                                          kTailBoxBytes, 128, 0);
          const uint64_t bd = ptx::make_desc(sB + j * atom_b + w * 32, 16, 1024, 2);
          ptx::mma_tf32(D, ad, bd, a.idesc, kk > 0 ? 1u : 0u);
        }
        ptx::mma_commit(empty0 + 8 * s);   // the stage may be refilled
        ptx::mma_commit(tfull0 + 8 * acc);  // the accumulator may be drained
        mmas = i + 1;
      }
    }
  } else {
    // group acc drains accumulator acc: the CTA's tiles acc, acc + kAcc, ...
    const int q = warp & 3, acc = (warp - 2) >> 2;
    const uint32_t lane_base = static_cast<uint32_t>(q * 32) << 16;
    const long long mstride = a.G * a.np_next;
    OutT *out = static_cast<OutT *>(a.out);
    long long i = acc;
    for (long long t = blockIdx.x + static_cast<long long>(acc) * gridDim.x; t < ntiles;
         t += static_cast<long long>(kAcc) * gridDim.x, i += kAcc) {
      const uint32_t aph = static_cast<uint32_t>((i / kAcc) & 1);
      // this lane's fiber and output offset (and eigenvalue) while the MMA runs
      const long long f = t * kFib + q * 32 + lane;
      const bool valid = f < a.rows;
      long long ob = 0;
      float ls = 0.f;
      if (valid) {
        const long long b = f / a.fib_per_b, fl = f - b * a.fib_per_b;
        const long long g = fl / a.n_next, inx = fl - g * a.n_next;
        ob = b * a.blk_out + g * a.np_next + inx;
        if (DIVIDE) ls = a.lam_s[fl];
      }
      if (!ptx::mbar_wait(tfull0 + 8 * acc, aph)) {
        ok = 0;
        break;
      }
      ptx::fence_after_sync();
      const uint32_t tbase = tmem + acc * kAccCols + lane_base;
      for (int c0 = 0; c0 < a.np; c0 += 64) {
        uint32_t r[64];
        const int nch = min(4, (a.np - c0) / 16);
#pragma unroll
        for (int cb = 0; cb < 4; ++cb)
          if (cb < nch) ptx::tmem_ld16_async(tbase + c0 + cb * 16, r + 16 * cb);
        ptx::tmem_wait_ld();
#pragma unroll
        for (int cb = 0; cb < 4; ++cb) ptx::reg_fence16(r + 16 * cb);
        if (valid) {
          OutT *po = out + ob + c0 * mstride;
          const int jn = min(64, a.n - c0);
#pragma unroll
          for (int j = 0; j < 64; ++j) {
            if (j < jn) {
              float v = __uint_as_float(r[j]);
              if (DIVIDE) v = __fdividef(v, s_lam_t[c0 + j] + ls);
              if (a.round_out) v = ptx::tf32_rna(v);
              store_val(po, v);
            }
            po += mstride;
          }
        }
      }
      ptx::fence_before_sync();
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(tempty0 + 8 * acc);
    }
  }
  __syncthreads();
  if (!ok) {
    // let this CTA's own copies and products land before its memory goes away
    if (warp == 0 && lane == 0) {
      *reinterpret_cast<volatile int *>(a.err) = 1;
      for (long long i = std::max(0LL, issued - S); i < issued; ++i)
        ptx::mbar_wait(full0 + 8 * static_cast<int>(i % S), static_cast<uint32_t>((i / S) & 1));
    }
    if (warp == 1 && lane == 0 && mmas > 0) {
      const long long i = mmas - 1;
      ptx::mbar_wait(tfull0 + 8 * static_cast<int>(i % kAcc), static_cast<uint32_t>((i / kAcc) & 1));
    }
  }
  ptx::fence_before_sync();
  __syncthreads();
  if (warp == 0) ptx::tmem_dealloc(tmem, kAcc * kAccCols);
}

// First-pass input: r (natural order, rows of n values) -> rows of np values
// rounded to TF32 (the padding is never read: the TMA unit zero-fills it).
template <typename IO>
__global__ void __launch_bounds__(256) pad_round_kernel(const IO *__restrict__ r, float *__restrict__ out,
                                                         unsigned total, unsigned n, unsigned np) {
  for (unsigned e = blockIdx.x * 256u + threadIdx.x; e < total; e += gridDim.x * 256u) {
    const unsigned row = e / n, k = e - row * n;
    float v;
    if constexpr (sizeof(IO) == 8)
      v = ptx::f64_to_f32_rn(r[e]);
    else
      v = r[e];
    out[static_cast<size_t>(row) * np + k] = ptx::tf32_rna(v);
  }
}

// K-major SW128 image of W (np rows x nkb * 32 K values): element (m, k) in
// atom k / 32 (np * 128 bytes each), row m (8-row groups 1024 bytes apart),
// 16-byte chunk (k % 32) / 4 XOR m % 8.  transpose: W[m][k] = U[k][m]
// (forward products), else U[m][k].  FP64 -> FP32 -> TF32 (ties away).
std::vector<uint8_t> sw128_image(const std::vector<double> &U, int n, int np, int nkb, bool transpose) {
  std::vector<uint8_t> img(static_cast<size_t>(nkb) * np * 128, 0);
  for (int m = 0; m < n; ++m)
    for (int k = 0; k < n; ++k) {
      const double w = transpose ? U[static_cast<size_t>(k) * n + m] : U[static_cast<size_t>(m) * n + k];
      const float f = static_cast<float>(w);
      uint32_t bits;
      std::memcpy(&bits, &f, 4);
      bits = (bits + 0x1000u) & 0xFFFFE000u;
      const int j = k / kBoxK, kk = k % kBoxK, c = kk / 4;
      const size_t off = static_cast<size_t>(j) * np * 128 + (m / 8) * 1024 + (m % 8) * 128 +
                         static_cast<size_t>((c ^ (m % 8)) * 16) + (kk % 4) * 4;
      std::memcpy(&img[off], &bits, 4);
    }
  return img;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (fn == nullptr) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// FP32 rows (n valid values, np apart) x rows; box 32 x 128, 128-byte swizzle,
// zero fill outside the tensor.
bool make_map(CUtensorMap &m, void *base, int n, int np, long long rows) {
  auto fn = encode_fn();
  if (fn == nullptr) return false;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(n), static_cast<cuuint64_t>(rows)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(np) * 4};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(kBoxK), static_cast<cuuint32_t>(kFib)};
  cuuint32_t estr[2] = {1, 1};
  return fn(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// FP32 rows as make_map, box 4 x 128 without swizzle (the no-swizzle tail).
bool make_tail_map(CUtensorMap &m, void *base, int n, int np, long long rows) {
  auto fn = encode_fn();
  if (fn == nullptr) return false;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(n), static_cast<cuuint64_t>(rows)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(np) * 4};
  cuuint32_t box[2] = {4u, static_cast<cuuint32_t>(kFib)};
  cuuint32_t estr[2] = {1, 1};
  return fn(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int ceil_to(int x, int m) { return (x + m - 1) / m * m; }

}  // namespace

struct RotFd {
  int d = 0, B = 0, sms = 0;
  int n[4] = {0, 0, 0, 0};
  long long N = 0;
  float *inter[2] = {nullptr, nullptr};
  const uint8_t *img_fwd[4] = {}, *img_bwd[4] = {};
  float *lam_t = nullptr, *lam_s = nullptr;
  int *err = nullptr;
  struct Pass {
    CUtensorMap map, tail;
    RotArgs args;
    size_t smem;
    int grid;
    bool divide, last;
  };
  std::vector<Pass> passes;
  unsigned pad_total = 0;
};

bool tc_fd_rot_eligible(int precision, int d, const int *n, int B) {
  if (precision != 1 || d < 1 || d > 3) return false;
  long long N = 1;
  for (int k = 0; k <= d; ++k) {
    if (n[k] < 1 || n[k] > 128) return false;
    N *= n[k];
  }
  // 32-bit element indices in the padding kernel (rows grow by at most 4/3)
  return static_cast<double>(B) * N * 4.0 / 3.0 < 4.0e9;
}

cudaError_t tc_fd_rot_create(RotFd *&out, std::vector<void *> &allocs, int d, const int *n, int B,
                             const std::vector<std::vector<double>> &U, const std::vector<std::vector<double>> &lam,
                             int *err_dev, std::string &err) {
  RotFd *f = new RotFd();
  out = f;
  f->d = d;
  f->B = B;
  f->err = err_dev;
  long long N = 1, Ns = 1;
  for (int k = 0; k <= d; ++k) {
    f->n[k] = n[k];
    N *= n[k];
    if (k < d) Ns *= n[k];
  }
  f->N = N;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&f->sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  auto alloc = [&](void **p, size_t bytes) {
    cudaError_t e2 = cudaMalloc(p, bytes + 16);
    if (e2 == cudaSuccess) allocs.push_back(*p);
    return e2;
  };
  // eigenvector images (forward U^T, backward U)
  int np_[4], npad[4], nkb[4];
  for (int k = 0; k <= d; ++k) {
    np_[k] = ceil_to(n[k], 16);
    npad[k] = ceil_to(n[k], 4);
    nkb[k] = (n[k] + kBoxK - 1) / kBoxK;
    for (int fwd = 0; fwd < 2; ++fwd) {
      const std::vector<uint8_t> img = sw128_image(U[k], n[k], np_[k], nkb[k], fwd == 1);
      void *p = nullptr;
      if ((e = alloc(&p, img.size())) != cudaSuccess) return e;
      if ((e = cudaMemcpy(p, img.data(), img.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
      (fwd ? f->img_fwd[k] : f->img_bwd[k]) = static_cast<const uint8_t *>(p);
    }
  }
  // intermediates: the padded layout of the largest pass input
  size_t inter = 0;
  for (int k = 0; k <= d; ++k) inter = std::max(inter, static_cast<size_t>(B) * static_cast<size_t>(N / n[k]) * npad[k]);
  for (int i = 0; i < 2; ++i) {
    void *p = nullptr;
    if ((e = alloc(&p, inter * sizeof(float))) != cudaSuccess) return e;
    f->inter[i] = static_cast<float *>(p);
  }
  // FP32 eigenvalues (the FP64 sums rounded once)
  std::vector<float> lt(n[d]), ls(Ns);
  for (int m = 0; m < n[d]; ++m) lt[m] = static_cast<float>(lam[d][m]);
  for (long long c = 0; c < Ns; ++c) {
    long long rem = c;
    double s = 0.0;
    for (int k = 0; k < d; ++k) {
      s += lam[k][rem % n[k]];
      rem /= n[k];
    }
    ls[c] = static_cast<float>(s);
  }
  void *p = nullptr;
  if ((e = alloc(&p, lt.size() * 4)) != cudaSuccess) return e;
  f->lam_t = static_cast<float *>(p);
  if ((e = alloc(&p, ls.size() * 4)) != cudaSuccess) return e;
  f->lam_s = static_cast<float *>(p);
  if ((e = cudaMemcpy(f->lam_t, lt.data(), lt.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess) return e;
  if ((e = cudaMemcpy(f->lam_s, ls.data(), ls.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess) return e;
  f->pad_total = static_cast<unsigned>(static_cast<long long>(B) * N);
  // passes: forward 0..d (U^T, division after the time product), backward 0..d (U)
  const int nprod = 2 * (d + 1);
  for (int st = 0; st < nprod; ++st) {
    const bool fwd = st <= d;
    const int k = fwd ? st : st - d - 1, kn = (k + 1) % (d + 1);
    const bool last = st == nprod - 1;
    RotFd::Pass ps{};
    RotArgs &a = ps.args;
    a.bimg = fwd ? f->img_fwd[k] : f->img_bwd[k];
    a.lam_t = f->lam_t;
    a.lam_s = f->lam_s;
    a.err = err_dev;
    a.fib_per_b = N / n[k];
    a.rows = static_cast<long long>(B) * a.fib_per_b;
    a.n = n[k];
    a.nkb = nkb[k];
    a.ksteps = (n[k] + 7) / 8;
    a.np = np_[k];
    a.n_next = n[kn];
    a.np_next = last ? n[kn] : npad[kn];
    a.G = a.fib_per_b / n[kn];
    a.blk_out = last ? N : (N / n[kn]) * npad[kn];
    a.round_out = last ? 0 : 1;
    a.bytes_b = static_cast<uint32_t>(nkb[k]) * np_[k] * 128;
    a.off_stage = a.bytes_b;  // a multiple of 1024 (np is a multiple of 16)
    a.idesc = ptx::idesc_tf32(kFib, np_[k]);
    // K groups: whole 32-value SW128 boxes and a tail of r <= 16 values in
    // 4-value boxes (2 per K step of 8; the TMA unit zero-fills past n_k).  The
    // stage size is a multiple of 1024 (an even number of 2048-byte tail boxes),
    // so every stage's SW128 atoms stay 1024-aligned.
    const int r = n[k] % kBoxK;
    a.full_atoms = (r > 0 && r <= kTailMax) ? n[k] / kBoxK : nkb[k];
    a.tail_boxes = (r > 0 && r <= kTailMax) ? 2 * ((r + 7) / 8) : 0;
    a.stage_bytes = static_cast<uint32_t>(a.full_atoms) * kBoxBytes + static_cast<uint32_t>(a.tail_boxes) * kTailBoxBytes;
    const size_t stage_bytes = a.stage_bytes;
    const size_t room = kSmemLimit - kStaticSmem - 1024 - a.bytes_b;
    a.stages = static_cast<int>(std::min<size_t>(kMaxStages, room / stage_bytes));
    if (a.stages < 2) {
      err = "TF32 preconditioner: pipeline stages do not fit in shared memory";
      return cudaErrorInvalidConfiguration;
    }
    ps.smem = 1024 + a.bytes_b + a.stages * stage_bytes;
    float *in = f->inter[(st + 1) % 2];
    if (!make_map(ps.map, in, n[k], npad[k], a.rows) || !make_tail_map(ps.tail, in, n[k], npad[k], a.rows)) {
      err = "TF32 preconditioner: cuTensorMapEncodeTiled failed";
      return cudaErrorInvalidConfiguration;
    }
    a.out = last ? nullptr : f->inter[st % 2];
    ps.divide = fwd && k == d;
    ps.last = last;
    const long long ntiles = (a.rows + kFib - 1) / kFib;
    ps.grid = static_cast<int>(std::min<long long>(ntiles, f->sms));
    f->passes.push_back(ps);
  }
  const size_t maxsm = std::max_element(f->passes.begin(), f->passes.end(), [](const RotFd::Pass &x,
                                                                                 const RotFd::Pass &y) {
                         return x.smem < y.smem;
                       })->smem;
  const int sm = static_cast<int>(maxsm);
  if ((e = raise_smem_limit(rot_kernel<float, false>, sm)) || (e = raise_smem_limit(rot_kernel<float, true>, sm)) ||
      (e = raise_smem_limit(rot_kernel<double, false>, sm)))
    return e;
  return cudaSuccess;
}

namespace {

template <typename IO>
cudaError_t launch_passes(RotFd *f, IO *z, cudaStream_t s);

}  // namespace

template <typename IO>
cudaError_t tc_fd_rot_apply(RotFd *f, const IO *r, IO *z, cudaStream_t s) {
  if (f == nullptr || f->passes.empty()) return cudaErrorNotReady;
  const unsigned total = f->pad_total;
  if (total > 0) {
    const unsigned g = std::min<unsigned>((total + 255) / 256, static_cast<unsigned>(f->sms) * 16);
    // the first pass reads inter[1]
    pad_round_kernel<IO><<<g, 256, 0, s>>>(r, f->inter[1], total, static_cast<unsigned>(f->n[0]),
                                           static_cast<unsigned>(ceil_to(f->n[0], 4)));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return launch_passes<IO>(f, z, s);
}

float *tc_fd_rot_padded_input(RotFd *f, int *n0, int *np0) {
  if (f == nullptr) return nullptr;
  if (n0) *n0 = f->n[0];
  if (np0) *np0 = ceil_to(f->n[0], 4);
  return f->inter[1];
}

cudaError_t tc_fd_rot_apply_padded(RotFd *f, float *z, cudaStream_t s) {
  if (f == nullptr || f->passes.empty()) return cudaErrorNotReady;
  return launch_passes<float>(f, z, s);
}

namespace {

template <typename IO>
cudaError_t launch_passes(RotFd *f, IO *z, cudaStream_t s) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  for (RotFd::Pass &ps : f->passes) {
    RotArgs a = ps.args;
    if (ps.last) a.out = z;
    if (ps.grid < 1) continue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(ps.grid));
    cfg.blockDim = dim3(kRotThreads);
    cfg.dynamicSmemBytes = ps.smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e;
    if (ps.last)
      e = cudaLaunchKernelEx(&cfg, rot_kernel<IO, false>, ps.map, ps.tail, a);
    else if (ps.divide)
      e = cudaLaunchKernelEx(&cfg, rot_kernel<float, true>, ps.map, ps.tail, a);
    else
      e = cudaLaunchKernelEx(&cfg, rot_kernel<float, false>, ps.map, ps.tail, a);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace

template cudaError_t tc_fd_rot_apply<float>(RotFd *, const float *, float *, cudaStream_t);
template cudaError_t tc_fd_rot_apply<double>(RotFd *, const double *, double *, cudaStream_t);

int tc_fd_rot_launches(const RotFd *f) { return f == nullptr ? 0 : static_cast<int>(f->passes.size()) + 1; }

void tc_fd_rot_destroy(RotFd *f) { delete f; }

}  // namespace stls
