// Fused tensor-core fast-diagonalization solve (Algorithm 1, steps 2-4) for
// d = 2 and d = 3 with BF16 operands and FP32 accumulation in tensor memory.
//
// The 2(d+1) mode products run in 2d - 1 launches instead of one per product:
//
//   slab_kernel (forward)   directions 1 and 2 of every 2D slice (fixed t[, i_3])
//   stream_kernel           direction 3, forward                       (d = 3)
//   stream_kernel<TIME>     time forward, division by the eigenvalue sum,
//                           time backward                              (fused)
//   stream_kernel           direction 3, backward                      (d = 3)
//   slab_kernel (backward)  directions 2 and 1 of every 2D slice
//
// so the backward products run in the order t, d, ..., 1 (the Kronecker
// factors commute; only the rounding points depend on the order).  Every
// product's FP32 result is rounded to BF16 before it is the next product's
// operand, and the intermediate tensors are BF16.
//
// Intermediate layout.  The forward slab kernel writes each slice transposed:
// Y[b][t][i_3][m_1][m_2] with the m_2 rows padded to P2 = ceil8(n_2) entries
// (zeros), so that every row is a whole number of 16-byte chunks.  For the
// streaming passes the tensor is then a 3D array (S, K, outer): S = n_1 * P2
// contiguous columns (direction 3 pass) or S3 = n_3 * S (time pass), K = the
// contracted direction, outer = the remaining index.  A streaming tile is
// 256 consecutive columns x all K rows; it is fetched by four TMA loads of
// 64-column boxes with 128-byte swizzle, which is the canonical MN-major
// operand layout of tcgen05 (rows = K, 128 bytes = 64 columns per row,
// 8-row groups 1024 B apart, 64-column atoms one box apart); rows K..kp-1 of a
// box lie outside the tensor and are zero-filled by the TMA unit.
//
// MMA orientation.  In every product the A operand is the eigenvector matrix
// (128 rows = output index, K-major image prepared on the host), the B operand
// is the data (N = columns), and the accumulator's TMEM lane is the output
// index of the contracted direction: warps whose 32 lanes hold valid rows run
// the epilogues.  The slab kernels chain two products per slice through
// shared memory: the first product's accumulator rows (lane = output index of
// direction a, columns = slice rows of direction b) are exactly K-major rows
// of the second product's A operand.
//
// Every mbarrier wait is bounded; on timeout the kernel records an error in
// host-mapped memory, lets its in-flight copies and MMAs finish (bounded) and
// frees its tensor memory.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "tc_fd.h"
#include "tc_ptx.cuh"

namespace stls {

namespace {

using bf16 = __nv_bfloat16;

constexpr int kThreads = 128;
constexpr int kSlabGroups = 3;         // independent warpgroup chains per slab CTA
constexpr int kSlabThreads = 128 * kSlabGroups;
constexpr int kSlabMaxN = 256;         // columns of the slab kernel's first product (MMA N)
constexpr int kTileN = 128;            // columns per streaming tile (MMA N)
constexpr int kAtomCols = 64;          // BF16 columns per 128-byte swizzle atom
constexpr int kAtoms = kTileN / kAtomCols;
constexpr int kStages = 3;             // input stages of a streaming kernel (outputs reuse them)
constexpr int kSmemLimit = 227 * 1024;   // per CTA
constexpr int kSmemPerSM = 228 * 1024;   // per SM
constexpr int kCtaReserve = 1024 + 256;  // reserved per CTA + static shared memory
constexpr int kStaticSmem = 256;         // barriers and flags (static shared memory)
constexpr uint32_t kStreamTmemCols = kTileN;
constexpr int kMaxCtasPerSM = 3;

__host__ __device__ inline int ceil_to(int x, int m) { return (x + m - 1) / m * m; }

__device__ __forceinline__ uint8_t *align1024(uint8_t *p) {
  const uint32_t a = ptx::smem_u32(p);
  return p + ((1024u - (a & 1023u)) & 1023u);
}

// Eight consecutive input values as FP32 (FP64 input: rounded to nearest even).
// The fallbacks take scalars, so the register arrays never need an address.
__device__ __forceinline__ float load1_f32(const float *p) { return *p; }
__device__ __forceinline__ float load1_f32(const double *p) { return ptx::f64_to_f32_rn(*p); }
__device__ __forceinline__ void load8_f32(const float *src, float *v) {
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = src[j];
}
__device__ __forceinline__ void load8_f32(const double *src, float *v) {
  bool ok = true;
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = ptx::f64_to_f32_fast(src[j], ok);
  if (!ok) {  // subnormal, huge, infinite or NaN results (rare)
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = ptx::f64_to_f32_hw(src[j]);
  }
}

__device__ __forceinline__ float out1(float v, float *) { return v; }
__device__ __forceinline__ double out1(float v, double *) { return ptx::f32_to_f64(v); }

// Sixteen FP32 accumulator values to the output type (FP64: exact widening).
__device__ __forceinline__ void to_out16(const uint32_t *r, float *o) {
#pragma unroll
  for (int e = 0; e < 16; ++e) o[e] = __uint_as_float(r[e]);
}
__device__ __forceinline__ void to_out16(const uint32_t *r, double *o) {
  bool ok = true;
#pragma unroll
  for (int e = 0; e < 16; ++e) o[e] = ptx::f32_to_f64_fast(__uint_as_float(r[e]), ok);
  if (!ok) {
#pragma unroll
    for (int e = 0; e < 16; ++e) o[e] = ptx::f32_to_f64_hw(__uint_as_float(r[e]));
  }
}

// ---------------------------------------------------------------------------
// Slab kernel: two spatial directions of G consecutive 2D slices per step.
//
// Input slice:  nb rows (direction b), each with the na values of direction a
//               contiguous (pitch in_pitch elements of InT).
// Output slice: na rows (output index of direction a), each with the nb output
//               values of direction b contiguous (pitch out_pitch of OutT;
//               out_cols values written per row).
// Product 1 contracts direction a:  D1[a'][g*Rb + b] = sum_a W_a[a'][a] X_g[b][a]
// Product 2 contracts direction b:  D2[a'][g*Rb + b'] = sum_b D1[a'][g*Rb + b] W_b[b'][b]
// Forward: (a, b) = (1, 2), InT = float|double, OutT = bf16 (transposed slice).
// Backward: (a, b) = (2, 1), InT = bf16 (transposed slice), OutT = float|double.
// ---------------------------------------------------------------------------
struct SlabArgs {
  const void *in;
  void *out;
  const uint8_t *imgA;  // W_a: ra rows x kpa (K-major, ra * 16 B per 8-wide K chunk)
  const uint8_t *imgB;  // W_b: Rb rows x Rb (K-major, Rb * 16 B per K chunk)
  long long nsl;        // slices
  int G;                // slices per step
  int na, nb, kpa, Rb;  // sizes; kpa = ceil16(na), Rb = ceil16(nb)
  float inv_nb;         // 1 / nb
  int ra;               // stored A rows = ceil8(na): rows ra..127 of an A operand are
                        // read from whatever follows (they only feed accumulator lanes >= na)
  int in_pitch, out_pitch, out_cols;
  uint32_t lbo_b1;      // K-chunk stride of the data operand: G * Rb * 16
  int off_A, off_B2, off_B1, off_A2, off_raw, off_out;  // buffers 0 and 1 follow each other
  int szA, szB2, szB1, szA2, szRaw, szOut;
  uint32_t idesc1, idesc2, tmem_cols, tmem_alloc;   // tmem_cols per group, tmem_alloc in all
  int groups;                                       // warpgroups with a chain (2 or 3)
  int *err;
};

// Warpgroups: the CTA's steps i = 0, 1, ... are dealt round-robin to its
// kSlabGroups (or 2, when the buffers of three do not fit) warpgroups; each runs
// the whole chain of its steps (input copy, conversion, product 1, epilogue 1,
// product 2, epilogue 2, output store) with its own buffers, tensor-memory
// columns, mbarriers and named barrier, so the chains of the groups overlap.
// Only the two eigenvector images are shared.
template <typename InT, typename OutT>
__global__ void __launch_bounds__(kSlabThreads, 1) slab_kernel(SlabArgs a) {
  extern __shared__ uint8_t smem_dyn[];
  __shared__ __align__(8) uint64_t bar_raw[kSlabGroups], bar_mma[kSlabGroups];
  __shared__ uint32_t tmem_holder;
  __shared__ int abort_flag;
  __shared__ uint16_t row_n[kSlabMaxN];  // data-operand row of input row g * nb + b
  uint8_t *sm = align1024(smem_dyn);
  const uint8_t *sA = sm + a.off_A, *sB2 = sm + a.off_B2;
  const int tid = threadIdx.x, warp = tid >> 5, wg = warp >> 2;
  const int lt = tid & 127;  // thread index within the warpgroup
  const int ngroups = a.groups;
  const long long nsteps = (a.nsl + a.G - 1) / a.G;
  const long long nloc = blockIdx.x < nsteps ? (nsteps - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const long long slice_in = static_cast<long long>(a.nb) * a.in_pitch * sizeof(InT);     // bytes
  const long long slice_out = static_cast<long long>(a.na) * a.out_pitch * sizeof(OutT);  // bytes
  const long long total_in = a.nsl * slice_in;
  const char *gin = static_cast<const char *>(a.in);
  char *gout = static_cast<char *>(a.out);
  const uint32_t tc = a.tmem_cols;  // accumulator columns per group

  for (int r = tid; r < a.G * a.nb; r += kSlabThreads) row_n[r] = static_cast<uint16_t>((r / a.nb) * a.Rb + r % a.nb);
  if (tid == 0) {
    for (int w = 0; w < kSlabGroups; ++w) {
      ptx::mbar_init(ptx::smem_u32(&bar_raw[w]), 1);
      ptx::mbar_init(ptx::smem_u32(&bar_mma[w]), 1);
    }
    ptx::mbar_init_fence();
    abort_flag = 0;
  }
  {
    const uint4 *srcA = reinterpret_cast<const uint4 *>(a.imgA);
    const uint4 *srcB = reinterpret_cast<const uint4 *>(a.imgB);
    for (int i = tid; i < a.szA / 16; i += kSlabThreads) reinterpret_cast<uint4 *>(sm + a.off_A)[i] = srcA[i];
    for (int i = tid; i < a.szB2 / 16; i += kSlabThreads) reinterpret_cast<uint4 *>(sm + a.off_B2)[i] = srcB[i];
    const uint4 zero = make_uint4(0, 0, 0, 0);
    // padding rows and K chunks of the data operands stay zero for the whole kernel
    for (int i = tid; i < ngroups * a.szB1 / 16; i += kSlabThreads) reinterpret_cast<uint4 *>(sm + a.off_B1)[i] = zero;
    for (int i = tid; i < ngroups * a.G * a.szA2 / 16; i += kSlabThreads)
      reinterpret_cast<uint4 *>(sm + a.off_A2)[i] = zero;
  }
  if (warp == 0) ptx::tmem_alloc(ptx::smem_u32(&tmem_holder), a.tmem_alloc);
  ptx::fence_proxy_async();
  ptx::fence_before_sync();
  __syncthreads();
  ptx::fence_after_sync();
  const uint32_t tmem = tmem_holder;
  const uint32_t lbo_a = static_cast<uint32_t>(a.ra) * 16;  // K-chunk stride of the A operands
  const int nch = a.Rb / 16;                                 // 16-column accumulator chunks per slice

  // Bounded wait; after any timeout every later wait returns at once, so that
  // all threads still reach every barrier and the kernel ends.
  auto wait = [&](uint64_t *bar, uint32_t parity) {
    if (*reinterpret_cast<volatile int *>(&abort_flag)) return;
    if (!ptx::mbar_wait(ptx::smem_u32(bar), parity)) {
      abort_flag = 1;
      *reinterpret_cast<volatile int *>(a.err) = 1;
    }
  };
  auto aborted = [&]() { return *reinterpret_cast<volatile int *>(&abort_flag) != 0; };
  // the bulk copy of a step's input covers [start & ~15, ceil16(end)), stopping
  // at end & ~15 where ceil16(end) would pass the end of the tensor
  auto bulk_end = [&](long long end) {
    const long long up = (end + 15) & ~15LL;
    return up <= total_in ? up : (end & ~15LL);
  };
  auto step_of = [&](long long i) { return static_cast<long long>(blockIdx.x) + i * gridDim.x; };

  if (wg < ngroups) {
    uint8_t *sRaw = sm + a.off_raw + wg * a.szRaw;
    uint8_t *sB1 = sm + a.off_B1 + wg * a.szB1;
    uint8_t *sA2 = sm + a.off_A2 + wg * a.G * a.szA2;
    uint8_t *sOut = sm + a.off_out + wg * a.szOut;
    uint64_t *braw = &bar_raw[wg], *bmma = &bar_mma[wg];
    const uint32_t tbuf = tmem + wg * tc;
    const uint32_t lane_base = static_cast<uint32_t>((warp & 3) * 32) << 16;
    const bool active = (warp & 3) * 32 < a.na;
    const bool valid = lt < a.na;
    uint32_t raw_phase = 0, mma_phase = 0;
    bool raw_pending = false;
    auto issue_raw = [&](long long i) {
      const long long s0 = step_of(i) * a.G;
      const long long gv = min(static_cast<long long>(a.G), a.nsl - s0);
      const long long start = s0 * slice_in, end = start + gv * slice_in;
      const long long b0 = start & ~15LL, b1 = bulk_end(end);
      if (b1 > b0) {
        ptx::mbar_expect_tx(ptx::smem_u32(braw), static_cast<uint32_t>(b1 - b0));
        ptx::bulk_g2s(ptx::smem_u32(sRaw), gin + b0, static_cast<uint32_t>(b1 - b0), ptx::smem_u32(braw));
        raw_pending = true;
      }
    };
    auto mma_wait = [&]() {
      wait(bmma, mma_phase);
      mma_phase ^= 1u;
    };
    if (lt == 0 && wg < nloc) issue_raw(wg);
    for (long long i = wg; i < nloc; i += ngroups) {
      const long long s0 = step_of(i) * a.G;
      const int gv = static_cast<int>(min(static_cast<long long>(a.G), a.nsl - s0));
      const long long start = s0 * slice_in, end = start + gv * slice_in;
      const long long b0 = start & ~15LL, b1 = bulk_end(end);
      if (b1 > b0) {
        wait(braw, raw_phase);
        raw_phase ^= 1u;
        raw_pending = false;
      }
      {
        // the last < 16 bytes of the tensor when the bulk copy stopped short of them
        const long long t0 = max(b1, b0);
        const int ntail = end > t0 ? static_cast<int>((end - t0) / static_cast<long long>(sizeof(InT))) : 0;
        if (lt < ntail) {
          const long long off = t0 + lt * static_cast<long long>(sizeof(InT));
          *reinterpret_cast<InT *>(sRaw + (off - b0)) = *reinterpret_cast<const InT *>(gin + off);
        }
      }
      ptx::named_sync(1 + wg, 128);
      {
        // items (row, 8-wide chunk), rows fastest across the threads, two items
        // per pass (both loaded before either is converted and stored)
        const int nrows = gv * a.nb;
        const int nchk = sizeof(InT) == 2 ? a.in_pitch / 8 : a.kpa / 8;
        const int nitems = nrows * nchk;  // items it = ch * nrows + row
        const uint8_t *raw = sRaw + (start - b0);
        auto do_item = [&](int ch, int row, bool load_only, float *v, uint4 *cp) {
          if constexpr (sizeof(InT) == 2) {
            if (load_only) {
              *cp = *reinterpret_cast<const uint4 *>(raw + (static_cast<size_t>(row) * a.in_pitch + ch * 8) * 2);
            } else {
              const int n = row_n[row];
              *reinterpret_cast<uint4 *>(sB1 + ch * a.lbo_b1 + (n >> 3) * 128 + (n & 7) * 16) = *cp;
            }
          } else {
            if (load_only) {
              const InT *src = reinterpret_cast<const InT *>(raw) + static_cast<size_t>(row) * a.in_pitch + ch * 8;
              if (ch * 8 + 8 <= a.na) {
                load8_f32(src, v);
              } else {
#pragma unroll
                for (int j = 0; j < 8; ++j) v[j] = ch * 8 + j < a.na ? load1_f32(src + j) : 0.f;
              }
            } else {
              const int n = row_n[row];
              uint4 pk;
              pk.x = ptx::pack_bf16(v[0], v[1]);
              pk.y = ptx::pack_bf16(v[2], v[3]);
              pk.z = ptx::pack_bf16(v[4], v[5]);
              pk.w = ptx::pack_bf16(v[6], v[7]);
              *reinterpret_cast<uint4 *>(sB1 + ch * a.lbo_b1 + (n >> 3) * 128 + (n & 7) * 16) = pk;
            }
          }
        };
        // item it = ch * nrows + row; (ch0, row0) for it and (ch1, row1) for it + 128,
        // both advanced by 256 items per pass without divisions
        int ch0 = lt / nrows, row0 = lt - ch0 * nrows;
        int ch1 = (lt + 128) / nrows, row1 = lt + 128 - ch1 * nrows;
        const int dch = 256 / nrows, drow = 256 - dch * nrows;
        for (int it = lt; it < nitems; it += 256) {
          float v0[8], v1[8];
          uint4 c0, c1;
          const bool two = it + 128 < nitems;
          do_item(ch0, row0, true, v0, &c0);
          if (two) do_item(ch1, row1, true, v1, &c1);
          do_item(ch0, row0, false, v0, &c0);
          if (two) do_item(ch1, row1, false, v1, &c1);
          ch0 += dch;
          row0 += drow;
          if (row0 >= nrows) {
            row0 -= nrows;
            ++ch0;
          }
          ch1 += dch;
          row1 += drow;
          if (row1 >= nrows) {
            row1 -= nrows;
            ++ch1;
          }
        }
      }
      ptx::fence_proxy_async();
      ptx::fence_before_sync();
      ptx::named_sync(1 + wg, 128);
      if (lt == 0) {
        ptx::fence_after_sync();
        // the input buffer is consumed: fetch this group's next step into it
        if (!aborted() && i + ngroups < nloc) issue_raw(i + ngroups);
        if (!aborted()) {
          const uint32_t a0 = ptx::smem_u32(sA), b0s = ptx::smem_u32(sB1);
          for (int kk = 0; kk < a.kpa / 16; ++kk) {
            const uint64_t ad = ptx::make_desc(a0 + kk * 2 * lbo_a, lbo_a, 128, 0);
            const uint64_t bd = ptx::make_desc(b0s + kk * 2 * a.lbo_b1, a.lbo_b1, 128, 0);
            ptx::mma_bf16(tbuf, ad, bd, a.idesc1, kk > 0 ? 1u : 0u);
          }
          ptx::mma_commit(ptx::smem_u32(bmma));
        }
      }
      mma_wait();
      ptx::fence_after_sync();
      // epilogue 1: accumulator row (lane) -> K-major row of product 2's A operand
      if (active) {
        const bool wr = lt < a.ra;
        for (int g = 0; g < gv; ++g) {
          uint8_t *dstA = sA2 + g * a.szA2 + (lt >> 3) * 128 + (lt & 7) * 16;
          for (int c4 = 0; c4 < nch; c4 += 4) {
            uint32_t r[64];
#pragma unroll
            for (int j = 0; j < 4; ++j)
              if (c4 + j < nch) ptx::tmem_ld16_async(tbuf + lane_base + g * a.Rb + (c4 + j) * 16, r + 16 * j);
            ptx::tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              if (c4 + j < nch) {
                ptx::reg_fence16(r + 16 * j);
                if (wr) {
#pragma unroll
                  for (int h = 0; h < 2; ++h) {
                    const uint32_t *v = r + 16 * j + 8 * h;
                    uint4 pk;
                    pk.x = ptx::pack_bf16(__uint_as_float(v[0]), __uint_as_float(v[1]));
                    pk.y = ptx::pack_bf16(__uint_as_float(v[2]), __uint_as_float(v[3]));
                    pk.z = ptx::pack_bf16(__uint_as_float(v[4]), __uint_as_float(v[5]));
                    pk.w = ptx::pack_bf16(__uint_as_float(v[6]), __uint_as_float(v[7]));
                    *reinterpret_cast<uint4 *>(dstA + (2 * (c4 + j) + h) * lbo_a) = pk;
                  }
                }
              }
            }
          }
        }
      }
      ptx::fence_proxy_async();
      ptx::fence_before_sync();
      if (lt == 0) ptx::bulk_wait_read<0>();  // this group's previous store has read its staging buffer
      ptx::named_sync(1 + wg, 128);
      if (lt == 0) {
        ptx::fence_after_sync();
        if (!aborted()) {
          const uint32_t a2 = ptx::smem_u32(sA2), b2 = ptx::smem_u32(sB2);
          const uint32_t lbo2 = static_cast<uint32_t>(a.Rb) * 16;
          for (int g = 0; g < gv; ++g) {
            for (int kk = 0; kk < a.Rb / 16; ++kk) {
              const uint64_t ad = ptx::make_desc(a2 + g * a.szA2 + kk * 2 * lbo_a, lbo_a, 128, 0);
              const uint64_t bd = ptx::make_desc(b2 + kk * 2 * lbo2, lbo2, 128, 0);
              ptx::mma_bf16(tbuf + g * a.Rb, ad, bd, a.idesc2, kk > 0 ? 1u : 0u);
            }
          }
          ptx::mma_commit(ptx::smem_u32(bmma));
        }
      }
      mma_wait();
      ptx::fence_after_sync();
      // epilogue 2: accumulator row (lane) = output row of the slice
      const long long ostart = s0 * slice_out, oend = ostart + gv * slice_out;
      const int ohead = static_cast<int>(ostart & 15);
      if (active) {
        for (int g = 0; g < gv; ++g) {
          const size_t rowoff = static_cast<size_t>(g * a.na + lt) * a.out_pitch;
          for (int c4 = 0; c4 < nch; c4 += 4) {
            uint32_t r[64];
#pragma unroll
            for (int j = 0; j < 4; ++j)
              if (c4 + j < nch) ptx::tmem_ld16_async(tbuf + lane_base + g * a.Rb + (c4 + j) * 16, r + 16 * j);
            ptx::tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const int cb = c4 + j;
              if (cb >= nch) continue;
              ptx::reg_fence16(r + 16 * j);
              if (!valid) continue;
              if constexpr (sizeof(OutT) == 2) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                  const int col = cb * 16 + 8 * h;
                  if (col < a.out_cols) {
                    const uint32_t *v = r + 16 * j + 8 * h;
                    uint4 pk;
                    pk.x = ptx::pack_bf16(__uint_as_float(v[0]), __uint_as_float(v[1]));
                    pk.y = ptx::pack_bf16(__uint_as_float(v[2]), __uint_as_float(v[3]));
                    pk.z = ptx::pack_bf16(__uint_as_float(v[4]), __uint_as_float(v[5]));
                    pk.w = ptx::pack_bf16(__uint_as_float(v[6]), __uint_as_float(v[7]));
                    *reinterpret_cast<uint4 *>(sOut + (rowoff + col) * 2) = pk;
                  }
                }
              } else {
                OutT *o = reinterpret_cast<OutT *>(sOut + ohead) + rowoff + cb * 16;
                if (cb * 16 + 16 <= a.out_cols) {
                  to_out16(r + 16 * j, o);
                } else {
#pragma unroll
                  for (int e = 0; e < 16; ++e)
                    if (cb * 16 + e < a.out_cols) o[e] = out1(__uint_as_float(r[16 * j + e]), o);
                }
              }
            }
          }
        }
      }
      ptx::fence_proxy_async();
      ptx::fence_before_sync();
      ptx::named_sync(1 + wg, 128);
      {
        // bulk store of the 16-byte aligned middle; plain stores for the ends
        const long long c0 = (ostart + 15) & ~15LL, c1 = oend & ~15LL;
        const long long base = ostart & ~15LL;  // global byte that maps to sOut[0]
        if (c1 > c0) {
          if (lt == 0) {
            ptx::bulk_s2g(gout + c0, ptx::smem_u32(sOut) + static_cast<uint32_t>(c0 - base),
                          static_cast<uint32_t>(c1 - c0));
            ptx::bulk_commit();
          }
          const int nh = static_cast<int>((c0 - ostart) / static_cast<long long>(sizeof(OutT)));
          const int nt = static_cast<int>((oend - c1) / static_cast<long long>(sizeof(OutT)));
          if (lt < nh) {
            const long long off = ostart + lt * static_cast<long long>(sizeof(OutT));
            *reinterpret_cast<OutT *>(gout + off) = *reinterpret_cast<const OutT *>(sOut + (off - base));
          } else if (lt >= 64 && lt < 64 + nt) {
            const long long off = c1 + (lt - 64) * static_cast<long long>(sizeof(OutT));
            *reinterpret_cast<OutT *>(gout + off) = *reinterpret_cast<const OutT *>(sOut + (off - base));
          }
        } else {
          const int ne = static_cast<int>((oend - ostart) / static_cast<long long>(sizeof(OutT)));
          for (int e = lt; e < ne; e += 128) {
            const long long off = ostart + e * static_cast<long long>(sizeof(OutT));
            *reinterpret_cast<OutT *>(gout + off) = *reinterpret_cast<const OutT *>(sOut + (off - base));
          }
        }
      }
    }
    if (lt == 0) {
      // in-flight stores, MMAs and input copies finish before the buffers go away
      ptx::bulk_wait<0>();
      if (raw_pending) ptx::mbar_wait(ptx::smem_u32(braw), raw_phase);
    }
  }
  ptx::fence_before_sync();
  __syncthreads();
  if (warp == 0) ptx::tmem_dealloc(tmem, a.tmem_alloc);
}

// ---------------------------------------------------------------------------
// Streaming kernel: one contracted direction with K = n rows (padded to kp),
// over a tensor (S, K, outer).  Tile = 256 columns x K rows of one outer index.
// D[m][c] = sum_k W[m][k] X[k][c].  TIME: W = U_t^T, then the division by
// lambda_t[m] + lambda_s[c] and the backward product with U_t on the same tile.
// ---------------------------------------------------------------------------
struct StreamArgs {
  const uint8_t *imgA, *imgA2;  // ra rows x kp, K-major (ra * 16 B per K chunk)
  const float *lam_t;           // TIME: >= 128 entries
  const float *lam_s;           // TIME: nct * 256 entries (padding 1)
  int n, kp, nouter, nct, ra;    // ra = ceil8(n) stored rows of the A images
  long long cols;               // S (or S3): columns of the tensor
  uint32_t atom_in;             // bytes per 64-column box: kp * 128
  int off_A, off_A2, off_stage, off_lam;  // off_lam: TIME, kTileN floats per stage
  int szA;
  uint32_t idesc;
  int *err;
};

template <bool TIME>
__global__ void __launch_bounds__(kThreads, 2)
    stream_kernel(const __grid_constant__ CUtensorMap tin, const __grid_constant__ CUtensorMap tout,
                  StreamArgs a) {
  extern __shared__ uint8_t smem_dyn[];
  __shared__ __align__(8) uint64_t bar_load[kStages];
  __shared__ __align__(8) uint64_t bar_mma;
  __shared__ uint32_t tmem_holder;
  __shared__ int ok;
  uint8_t *sm = align1024(smem_dyn);
  uint8_t *sA = sm + a.off_A, *sA2 = sm + a.off_A2;
  uint8_t *stage0 = sm + a.off_stage;
  const uint32_t sz_stage = kAtoms * a.atom_in;
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t lb0 = ptx::smem_u32(&bar_load[0]), mb = ptx::smem_u32(&bar_mma);
  const long long ntiles = static_cast<long long>(a.nouter) * a.nct;

  if (tid == 0) {
    for (int k = 0; k < kStages; ++k) ptx::mbar_init(lb0 + 8 * k, 1);
    ptx::mbar_init(mb, 1);
    ptx::mbar_init_fence();
    ok = 1;
  }
  {
    const uint4 zero = make_uint4(0, 0, 0, 0);
    for (uint32_t i = tid; i < kStages * sz_stage / 16; i += kThreads) reinterpret_cast<uint4 *>(stage0)[i] = zero;
    const uint4 *src = reinterpret_cast<const uint4 *>(a.imgA);
    for (int i = tid; i < a.szA / 16; i += kThreads) reinterpret_cast<uint4 *>(sA)[i] = src[i];
    if (TIME) {
      const uint4 *src2 = reinterpret_cast<const uint4 *>(a.imgA2);
      for (int i = tid; i < a.szA / 16; i += kThreads) reinterpret_cast<uint4 *>(sA2)[i] = src2[i];
    }
  }
  if (warp == 0) ptx::tmem_alloc(ptx::smem_u32(&tmem_holder), kStreamTmemCols);
  ptx::fence_proxy_async();
  ptx::fence_before_sync();
  __syncthreads();
  ptx::fence_after_sync();
  const uint32_t tmem = tmem_holder;
  const uint32_t lane_base = static_cast<uint32_t>(warp * 32) << 16;
  const uint32_t lbo_a = static_cast<uint32_t>(a.ra) * 16;

  // boxes of a tile that start inside the tensor (the rest of a ragged last
  // tile is never stored, and its stale, finite columns never mix with others)
  auto boxes = [&](int c0) {
    const long long left = a.cols - c0;
    return static_cast<int>(min(static_cast<long long>(kAtoms), (left + kAtomCols - 1) / kAtomCols));
  };
  auto issue_load = [&](long long t, int s) {
    const int o = static_cast<int>(t / a.nct), c0 = static_cast<int>(t % a.nct) * kTileN;
    const uint32_t bar = lb0 + 8 * s, dst = ptx::smem_u32(stage0) + s * sz_stage;
    const int nb = boxes(c0);
    ptx::mbar_expect_tx(bar, nb * a.atom_in + (TIME ? kTileN * 4 : 0));
    for (int at = 0; at < nb; ++at) ptx::tma_load_3d(dst + at * a.atom_in, &tin, c0 + at * kAtomCols, 0, o, bar);
    // the tile's lambda_s (padded to whole tiles) travels with it
    if (TIME) ptx::bulk_g2s(ptx::smem_u32(sm + a.off_lam) + s * kTileN * 4, a.lam_s + c0, kTileN * 4, bar);
  };
  auto issue_mma = [&](const uint8_t *A, int s) {
    const uint32_t a0 = ptx::smem_u32(A), b0 = ptx::smem_u32(stage0) + s * sz_stage;
    for (int kk = 0; kk < a.kp / 16; ++kk) {
      const uint64_t ad = ptx::make_desc(a0 + kk * 2 * lbo_a, lbo_a, 128, 0);
      const uint64_t bd = ptx::make_desc(b0 + kk * 2048, a.atom_in, 1024, 2);
      ptx::mma_bf16(tmem, ad, bd, a.idesc, kk > 0 ? 1u : 0u);
    }
    ptx::mma_commit(mb);
  };
  // 64 columns of this thread's accumulator row, one wait for the four loads
  auto load_half = [&](int half, uint32_t *r) {
#pragma unroll
    for (int cb = 0; cb < 4; ++cb) ptx::tmem_ld16_async(tmem + lane_base + half * 64 + cb * 16, r + 16 * cb);
    ptx::tmem_wait_ld();
#pragma unroll
    for (int cb = 0; cb < 4; ++cb) ptx::reg_fence16(r + 16 * cb);
  };
  // 128-byte swizzle: 16-byte chunk q of row m of a box lives at chunk q ^ (m % 8)
  auto box_addr = [](uint8_t *box, int m, int q) { return box + (m >> 3) * 1024 + (m & 7) * 128 + ((q ^ (m & 7)) << 4); };

  uint32_t mma_phase = 0;
  bool mma_pending = false;                        // thread 0: for the error path
  bool load_pending[kStages] = {};
  uint32_t load_phase[kStages] = {};
  if (tid == 0) {
    for (int i = 0; i < 2; ++i) {
      const long long t = blockIdx.x + static_cast<long long>(i) * gridDim.x;
      if (t < ntiles) {
        issue_load(t, i);
        load_pending[i] = true;
      }
    }
  }
  int it = 0;
  const bool active = warp * 32 < a.n;
  const bool valid = tid < a.n;
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
    const int s = it % kStages;
    const int o = static_cast<int>(t / a.nct), c0 = static_cast<int>(t % a.nct) * kTileN;
    uint8_t *stage = stage0 + s * sz_stage;
    if (ptx::mbar_wait(lb0 + 8 * s, load_phase[s])) {
      load_phase[s] ^= 1u;
      load_pending[s] = false;
    } else {
      ok = 0;
    }
    __syncthreads();
    if (!ok) break;
    if (tid == 0) {
      ptx::fence_after_sync();
      issue_mma(sA, s);
      mma_pending = true;
    }
    if (ptx::mbar_wait(mb, mma_phase)) {
      mma_phase ^= 1u;
      mma_pending = false;
    } else {
      ok = 0;
    }
    ptx::fence_after_sync();
    if (TIME) {
      // division by the eigenvalue sum; the quotient (BF16) replaces the tile
      // in place as the B operand of the backward time product
      if (active) {
        const float lt = valid ? a.lam_t[tid] : 1.f;
        for (int half = 0; half < kTileN / 64; ++half) {
          uint32_t r[64];
          load_half(half, r);
          if (!valid) continue;
          const float4 *ls4 = reinterpret_cast<const float4 *>(sm + a.off_lam + s * kTileN * 4) + half * 16;
#pragma unroll
          for (int qq = 0; qq < 8; ++qq) {
            const int q = half * 8 + qq;
            const float4 l0 = ls4[2 * qq], l1 = ls4[2 * qq + 1];
            const uint32_t *u = r + 8 * qq;
            uint4 pk;
            pk.x = ptx::pack_bf16(__fdividef(__uint_as_float(u[0]), lt + l0.x), __fdividef(__uint_as_float(u[1]), lt + l0.y));
            pk.y = ptx::pack_bf16(__fdividef(__uint_as_float(u[2]), lt + l0.z), __fdividef(__uint_as_float(u[3]), lt + l0.w));
            pk.z = ptx::pack_bf16(__fdividef(__uint_as_float(u[4]), lt + l1.x), __fdividef(__uint_as_float(u[5]), lt + l1.y));
            pk.w = ptx::pack_bf16(__fdividef(__uint_as_float(u[6]), lt + l1.z), __fdividef(__uint_as_float(u[7]), lt + l1.w));
            *reinterpret_cast<uint4 *>(box_addr(stage + (q >> 3) * a.atom_in, tid, q & 7)) = pk;
          }
        }
      }
      ptx::fence_proxy_async();
      ptx::fence_before_sync();
      __syncthreads();
      if (tid == 0) {
        ptx::fence_after_sync();
        issue_mma(sA2, s);
        mma_pending = true;
      }
      if (ptx::mbar_wait(mb, mma_phase)) {
        mma_phase ^= 1u;
        mma_pending = false;
      } else {
        ok = 0;
      }
      ptx::fence_after_sync();
    }
    // the products have read the stage: the output rows go into it (same
    // swizzled box layout) and the TMA store reads them from there
    uint8_t *stg = stage;
    if (active) {
      for (int half = 0; half < kTileN / 64; ++half) {
        uint32_t r[64];
        load_half(half, r);
        if (!valid) continue;
#pragma unroll
        for (int qq = 0; qq < 8; ++qq) {
          const int q = half * 8 + qq;
          const uint32_t *u = r + 8 * qq;
          uint4 pk;
          pk.x = ptx::pack_bf16(__uint_as_float(u[0]), __uint_as_float(u[1]));
          pk.y = ptx::pack_bf16(__uint_as_float(u[2]), __uint_as_float(u[3]));
          pk.z = ptx::pack_bf16(__uint_as_float(u[4]), __uint_as_float(u[5]));
          pk.w = ptx::pack_bf16(__uint_as_float(u[6]), __uint_as_float(u[7]));
          *reinterpret_cast<uint4 *>(box_addr(stg + (q >> 3) * a.atom_in, tid, q & 7)) = pk;
        }
      }
    }
    ptx::fence_proxy_async();
    ptx::fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      const uint32_t src = ptx::smem_u32(stg);
      const int nb = boxes(c0);
      for (int at = 0; at < nb; ++at) ptx::tma_store_3d(&tout, c0 + at * kAtomCols, 0, o, src + at * a.atom_in);
      ptx::bulk_commit();
      // fetch two tiles ahead into the stage of the previous tile, once that
      // tile's store has read it (at most this tile's store still reads)
      const long long tn = t + 2LL * gridDim.x;
      if (ok && !mma_pending && tn < ntiles) {
        const int sn = (it + 2) % kStages;
        ptx::bulk_wait_read<1>();
        issue_load(tn, sn);
        load_pending[sn] = true;
      }
    }
  }
  if (tid == 0) {
    ptx::bulk_wait<0>();
    if (!ok) {
      *reinterpret_cast<volatile int *>(a.err) = 1;
      for (int k = 0; k < kStages; ++k)
        if (load_pending[k]) ptx::mbar_wait(lb0 + 8 * k, load_phase[k]);
      if (mma_pending) ptx::mbar_wait(mb, mma_phase);
    }
  }
  ptx::fence_before_sync();
  __syncthreads();
  if (warp == 0) ptx::tmem_dealloc(tmem, kStreamTmemCols);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

// K-major no-swizzle image of W (rows x kp): element (m, k) at
// (k / 8) * (rows * 16) + (m / 8) * 128 + (m % 8) * 16 + (k % 8) * 2.
// transpose: W[m][k] = U[k][m] (forward products); else U[m][k].
std::vector<uint8_t> kmajor_image(const std::vector<double> &U, int n, int rows, int kp, bool transpose) {
  const size_t lbo = static_cast<size_t>(rows) * 16;
  std::vector<uint8_t> img(static_cast<size_t>(kp / 8) * lbo, 0);
  for (int m = 0; m < n; ++m)
    for (int k = 0; k < n; ++k) {
      const double w = transpose ? U[static_cast<size_t>(k) * n + m] : U[static_cast<size_t>(m) * n + k];
      const size_t off = static_cast<size_t>(k / 8) * lbo + (m / 8) * 128 + (m % 8) * 16 + (k % 8) * 2;
      const bf16 h = __float2bfloat16_rn(static_cast<float>(w));
      memcpy(&img[off], &h, 2);
    }
  return img;
}

struct SlabPlan {
  SlabArgs args{};
  int smem = 0, grid = 0;
};

struct StreamPlan {
  StreamArgs args{};
  CUtensorMap tin{}, tout{};
  int smem = 0, grid = 0;
};

}  // namespace

struct FusedFd {
  int d = 0, B = 0;
  int n1 = 0, n2 = 0, n3 = 1, nt = 0, P2 = 0;
  long long S = 0, S3 = 0, nsl = 0, Y = 0;
  bf16 *ya = nullptr, *yb = nullptr;
  SlabPlan fwd32, fwd64, bwd32, bwd64;
  StreamPlan mid_f, mid_b, time;
  int sms = 0;
};

namespace {

template <typename T>
cudaError_t falloc(std::vector<void *> &allocs, T **p, size_t count) {
  void *v = nullptr;
  cudaError_t e = cudaMalloc(&v, count * sizeof(T) + 16);
  if (e != cudaSuccess) return e;
  allocs.push_back(v);
  *p = static_cast<T *>(v);
  return cudaSuccess;
}

cudaError_t upload_img(std::vector<void *> &allocs, const std::vector<uint8_t> &img, const uint8_t **dst) {
  uint8_t *p = nullptr;
  cudaError_t e = falloc(allocs, &p, img.size());
  if (e != cudaSuccess) return e;
  *dst = p;
  return cudaMemcpy(p, img.data(), img.size(), cudaMemcpyHostToDevice);
}

int up1024(long long x) { return static_cast<int>((x + 1023) / 1024 * 1024); }

// CTAs of `smem` dynamic bytes that fit on one SM (at most kMaxCtasPerSM).
int ctas_per_sm(int smem) { return std::max(1, std::min(kMaxCtasPerSM, kSmemPerSM / (smem + kCtaReserve))); }

// Slack after a compact A operand: an M = 128 MMA reads rows ra..127 of the
// last K chunk past its end.
int a_slack(int ra) { return (128 - ra) * 16; }

// Shared-memory layout of a slab kernel with G slices per step and `groups`
// warpgroup chains (one set of per-step buffers each); returns the dynamic size
// (0 if it does not fit).
int slab_layout(SlabArgs &s, int G, int groups, size_t in_size, size_t out_size) {
  auto up16 = [](long long x) { return static_cast<int>((x + 15) / 16 * 16); };
  s.G = G;
  s.groups = groups;
  s.szA = s.kpa / 8 * s.ra * 16;
  s.szB2 = s.Rb / 8 * s.Rb * 16;
  s.lbo_b1 = static_cast<uint32_t>(G * s.Rb * 16);
  s.szB1 = s.kpa / 8 * static_cast<int>(s.lbo_b1);
  s.szA2 = s.Rb / 8 * s.ra * 16;
  s.szRaw = up16(static_cast<long long>(G) * s.nb * s.in_pitch * in_size + 32);  // + head and tail
  s.szOut = up16(static_cast<long long>(G) * s.na * s.out_pitch * out_size + 16);
  int off = 0;
  s.off_A = off;
  off += up1024(s.szA + a_slack(s.ra));
  s.off_B2 = off;
  off += up1024(s.szB2);
  s.off_B1 = off;
  off += up1024(static_cast<long long>(groups) * s.szB1);
  s.off_A2 = off;
  off += up1024(static_cast<long long>(groups) * G * s.szA2 + a_slack(s.ra));
  s.off_raw = off;
  off += up1024(static_cast<long long>(groups) * s.szRaw);
  s.off_out = off;
  off += up1024(static_cast<long long>(groups) * s.szOut);
  const int total = off + 1024;  // alignment of the dynamic base
  return total + kStaticSmem <= kSmemLimit ? total : 0;
}

// Three warpgroup chains if their buffers fit, else two; then the largest G
// (G * Rb <= 256, and <= 128 with three chains: their accumulators share the
// 512 tensor-memory columns) that fits.
template <typename InT, typename OutT>
cudaError_t plan_slab(SlabPlan &pl, SlabArgs base, long long nsl, int sms) {
  for (int groups = kSlabGroups; groups >= 2; --groups) {
    const int maxn = groups == 3 ? 128 : kSlabMaxN;
    const int gmax = static_cast<int>(std::min<long long>(maxn / base.Rb, nsl));
    for (int G = gmax; G >= 1; --G) {
      SlabArgs s = base;
      const int smem = slab_layout(s, G, groups, sizeof(InT), sizeof(OutT));
      if (smem == 0) continue;
      s.nsl = nsl;
      s.inv_nb = 1.0f / static_cast<float>(s.nb);
      s.idesc1 = ptx::idesc_bf16(128, G * s.Rb, 0);
      s.idesc2 = ptx::idesc_bf16(128, s.Rb, 0);
      uint32_t cols = 32;
      while (cols < static_cast<uint32_t>(G * s.Rb)) cols *= 2;
      s.tmem_cols = cols;
      uint32_t alloc = 32;
      while (alloc < static_cast<uint32_t>(groups) * cols) alloc *= 2;
      if (alloc > 512) continue;
      s.tmem_alloc = alloc;
      pl.args = s;
      pl.smem = smem;
      const long long nsteps = (nsl + G - 1) / G;
      pl.grid = static_cast<int>(std::min<long long>(nsteps, sms));
      return raise_smem_limit(slab_kernel<InT, OutT>, smem);
    }
  }
  return cudaErrorInvalidConfiguration;
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

// BF16 tensor (cols, rows, outer) with cols contiguous; box 64 x box_rows x 1, 128-byte swizzle.
bool make_map(CUtensorMap &m, void *base, long long cols, int rows, long long outer, int box_rows) {
  auto fn = encode_fn();
  if (fn == nullptr) return false;
  cuuint64_t dims[3] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows), static_cast<cuuint64_t>(outer)};
  cuuint64_t strides[2] = {static_cast<cuuint64_t>(cols) * 2, static_cast<cuuint64_t>(cols) * rows * 2};
  cuuint32_t box[3] = {static_cast<cuuint32_t>(kAtomCols), static_cast<cuuint32_t>(box_rows), 1};
  cuuint32_t estr[3] = {1, 1, 1};
  return fn(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <bool TIME>
cudaError_t plan_stream(StreamPlan &pl, int n, long long cols, long long outer, void *in, void *out, int sms,
                        std::string &err) {
  StreamArgs &s = pl.args;
  s.n = n;
  s.kp = ceil_to(n, 16);
  s.ra = ceil_to(n, 8);
  s.nouter = static_cast<int>(outer);
  s.nct = static_cast<int>((cols + kTileN - 1) / kTileN);
  s.cols = cols;
  s.atom_in = static_cast<uint32_t>(s.kp) * 128;
  s.szA = s.kp / 8 * s.ra * 16;
  int off = 0;
  s.off_stage = off;  // stages first: every operand address stays inside the allocation
  off += kStages * kAtoms * static_cast<int>(s.atom_in);
  s.off_A = off;
  off += up1024(s.szA + a_slack(s.ra));
  s.off_A2 = off;
  if (TIME) off += up1024(s.szA + a_slack(s.ra));
  s.off_lam = off;
  if (TIME) off += kStages * kTileN * 4;
  pl.smem = off + 1024;
  if (pl.smem + kStaticSmem > kSmemLimit) {
    err = "tensor-core preconditioner: streaming tile does not fit in shared memory";
    return cudaErrorInvalidConfiguration;
  }
  s.idesc = ptx::idesc_bf16(128, kTileN, 1);
  if (!make_map(pl.tin, in, cols, n, outer, s.kp) || !make_map(pl.tout, out, cols, n, outer, n)) {
    err = "tensor-core preconditioner: cuTensorMapEncodeTiled failed";
    return cudaErrorInvalidConfiguration;
  }
  const long long ntiles = outer * s.nct;
  pl.grid = static_cast<int>(std::min<long long>(ntiles, static_cast<long long>(sms) * ctas_per_sm(pl.smem)));
  return raise_smem_limit(stream_kernel<TIME>, pl.smem);
}

}  // namespace

bool tc_fd_fused_eligible(int precision, int d, const int *n) {
  if (precision != 2 || (d != 2 && d != 3)) return false;
  for (int k = 0; k <= d; ++k)
    if (n[k] < 1 || n[k] > 128) return false;
  return true;
}

cudaError_t tc_fd_fused_create(FusedFd *&out, std::vector<void *> &allocs, int d, const int *n, int B,
                               const std::vector<std::vector<double>> &U, const std::vector<std::vector<double>> &lam,
                               int *err_dev, std::string &err) {
  FusedFd *f = new FusedFd();
  out = f;
  f->d = d;
  f->B = B;
  f->n1 = n[0];
  f->n2 = n[1];
  f->n3 = d == 3 ? n[2] : 1;
  f->nt = n[d];
  f->P2 = ceil_to(f->n2, 8);
  f->S = static_cast<long long>(f->n1) * f->P2;
  f->S3 = f->S * f->n3;
  f->nsl = static_cast<long long>(B) * f->nt * f->n3;
  f->Y = f->nsl * f->S;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&f->sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = falloc(allocs, &f->ya, static_cast<size_t>(f->Y))) != cudaSuccess) return e;
  if ((e = falloc(allocs, &f->yb, static_cast<size_t>(f->Y))) != cudaSuccess) return e;

  // slab kernels
  const int kp1 = ceil_to(f->n1, 16), kp2 = ceil_to(f->n2, 16);
  {
    SlabArgs s{};
    s.na = f->n1;
    s.nb = f->n2;
    s.ra = ceil_to(f->n1, 8);
    s.kpa = kp1;
    s.Rb = kp2;
    s.in_pitch = f->n1;
    s.out_pitch = f->P2;
    s.out_cols = f->P2;
    s.err = err_dev;
    if ((e = upload_img(allocs, kmajor_image(U[0], f->n1, ceil_to(f->n1, 8), kp1, true), &s.imgA)) != cudaSuccess) return e;
    if ((e = upload_img(allocs, kmajor_image(U[1], f->n2, kp2, kp2, true), &s.imgB)) != cudaSuccess) return e;
    if ((e = plan_slab<float, bf16>(f->fwd32, s, f->nsl, f->sms)) != cudaSuccess) return e;
    if ((e = plan_slab<double, bf16>(f->fwd64, s, f->nsl, f->sms)) != cudaSuccess) return e;
  }
  {
    SlabArgs s{};
    s.na = f->n2;
    s.nb = f->n1;
    s.ra = ceil_to(f->n2, 8);
    s.kpa = kp2;
    s.Rb = kp1;
    s.in_pitch = f->P2;
    s.out_pitch = f->n1;
    s.out_cols = f->n1;
    s.err = err_dev;
    if ((e = upload_img(allocs, kmajor_image(U[1], f->n2, ceil_to(f->n2, 8), kp2, false), &s.imgA)) != cudaSuccess) return e;
    if ((e = upload_img(allocs, kmajor_image(U[0], f->n1, kp1, kp1, false), &s.imgB)) != cudaSuccess) return e;
    if ((e = plan_slab<bf16, float>(f->bwd32, s, f->nsl, f->sms)) != cudaSuccess) return e;
    if ((e = plan_slab<bf16, double>(f->bwd64, s, f->nsl, f->sms)) != cudaSuccess) return e;
  }
  // direction-3 passes: tensor (S, n3, B * nt); forward reads ya writes yb, backward the same
  if (d == 3) {
    const int kp3 = ceil_to(f->n3, 16);
    for (int dirn = 0; dirn < 2; ++dirn) {
      StreamPlan &pl = dirn == 0 ? f->mid_f : f->mid_b;
      pl.args.err = err_dev;
      if ((e = upload_img(allocs, kmajor_image(U[2], f->n3, ceil_to(f->n3, 8), kp3, dirn == 0), &pl.args.imgA)) != cudaSuccess)
        return e;
      if ((e = plan_stream<false>(pl, f->n3, f->S, static_cast<long long>(B) * f->nt, f->ya, f->yb, f->sms, err)) !=
          cudaSuccess)
        return e;
    }
  }
  // time pass: tensor (S3, nt, B); reads the forward direction-3 output
  {
    StreamPlan &pl = f->time;
    StreamArgs &s = pl.args;
    s.err = err_dev;
    const int kpt = ceil_to(f->nt, 16);
    if ((e = upload_img(allocs, kmajor_image(U[d], f->nt, ceil_to(f->nt, 8), kpt, true), &s.imgA)) != cudaSuccess) return e;
    if ((e = upload_img(allocs, kmajor_image(U[d], f->nt, ceil_to(f->nt, 8), kpt, false), &s.imgA2)) != cudaSuccess) return e;
    bf16 *tin = d == 3 ? f->yb : f->ya, *tout = d == 3 ? f->ya : f->yb;
    if ((e = plan_stream<true>(pl, f->nt, f->S3, B, tin, tout, f->sms, err)) != cudaSuccess) return e;
    // eigenvalues rounded once to FP32; lambda_s in the column order of the time pass
    std::vector<float> lt(128, 1.f);
    for (int i = 0; i < f->nt; ++i) lt[i] = static_cast<float>(lam[d][i]);
    std::vector<float> ls(static_cast<size_t>(s.nct) * kTileN, 1.f);
    for (int i3 = 0; i3 < f->n3; ++i3)
      for (int m1 = 0; m1 < f->n1; ++m1)
        for (int m2 = 0; m2 < f->n2; ++m2) {
          const double v = lam[0][m1] + lam[1][m2] + (d == 3 ? lam[2][i3] : 0.0);
          ls[(static_cast<size_t>(i3) * f->n1 + m1) * f->P2 + m2] = static_cast<float>(v);
        }
    float *dlt = nullptr, *dls = nullptr;
    if ((e = falloc(allocs, &dlt, lt.size())) != cudaSuccess) return e;
    if ((e = falloc(allocs, &dls, ls.size())) != cudaSuccess) return e;
    if ((e = cudaMemcpy(dlt, lt.data(), 4 * lt.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
    if ((e = cudaMemcpy(dls, ls.data(), 4 * ls.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
    s.lam_t = dlt;
    s.lam_s = dls;
  }
  return cudaSuccess;
}

int tc_fd_fused_launches(const FusedFd *f) { return 2 * f->d - 1; }

template <typename IO>
cudaError_t tc_fd_fused_apply(FusedFd *f, const IO *r, IO *z, cudaStream_t st) {
  const SlabPlan &pf = sizeof(IO) == 8 ? f->fwd64 : f->fwd32;
  const SlabPlan &pb = sizeof(IO) == 8 ? f->bwd64 : f->bwd32;
  SlabArgs af = pf.args, ab = pb.args;
  af.in = r;
  af.out = f->ya;
  slab_kernel<IO, bf16><<<pf.grid, kSlabThreads, pf.smem, st>>>(af);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (f->d == 3) {
    stream_kernel<false><<<f->mid_f.grid, kThreads, f->mid_f.smem, st>>>(f->mid_f.tin, f->mid_f.tout, f->mid_f.args);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  stream_kernel<true><<<f->time.grid, kThreads, f->time.smem, st>>>(f->time.tin, f->time.tout, f->time.args);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (f->d == 3) {
    stream_kernel<false><<<f->mid_b.grid, kThreads, f->mid_b.smem, st>>>(f->mid_b.tin, f->mid_b.tout, f->mid_b.args);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  ab.in = f->yb;
  ab.out = z;
  slab_kernel<bf16, IO><<<pb.grid, kSlabThreads, pb.smem, st>>>(ab);
  return cudaGetLastError();
}

template cudaError_t tc_fd_fused_apply<float>(FusedFd *, const float *, float *, cudaStream_t);
template cudaError_t tc_fd_fused_apply<double>(FusedFd *, const double *, double *, cudaStream_t);

void tc_fd_fused_destroy(FusedFd *f) { delete f; }

namespace {

__global__ void round_bf16_kernel(const double *x, double *y, long long n) {
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const float f = ptx::f64_to_f32_rn(x[i]);
    y[i] = ptx::f32_to_f64(__bfloat162float(__float2bfloat16_rn(f)));
  }
}

}  // namespace

cudaError_t round_bf16_launch(const double *x, double *y, long long n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const long long blocks = std::min<long long>((n + 255) / 256, 152LL * 16);
  round_bf16_kernel<<<static_cast<unsigned>(blocks), 256, 0, s>>>(x, y, n);
  return cudaGetLastError();
}

}  // namespace stls
