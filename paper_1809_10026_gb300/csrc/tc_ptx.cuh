// Inline-PTX helpers for the sm_103a tensor-core kernels: shared-memory matrix
// descriptors, tcgen05 MMA / commit / tensor-memory loads, mbarriers with
// bounded waits, bulk and tensor (TMA) copies.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

namespace stls {
namespace ptx {

// A wait on an mbarrier suspends the thread (try_wait with a suspend-time hint)
// instead of spinning, so that waiting warps leave the issue slots to the
// working ones; it is declared failed after kWaitLimitNs of global time.
constexpr uint32_t kSuspendHintNs = 10000000u;
constexpr unsigned long long kWaitLimitNs = 4000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// tcgen05 shared-memory matrix descriptor: start address, leading and stride
// byte offsets (all >> 4), descriptor version 1 (bit 46), swizzle mode in bits
// 61-63 (0 none, 2 = 128-byte swizzle).
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo, uint32_t swizzle) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr >> 4) & 0x3FFFu);
  d |= static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16;
  d |= static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32;
  d |= 1ull << 46;
  d |= static_cast<uint64_t>(swizzle & 7u) << 61;
  return d;
}

// D[tmem] (+)= A * B, BF16 operands, FP32 accumulator, issued by one thread.
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

// D[tmem] (+)= A * B, TF32 operands (the top 19 bits of each FP32 operand),
// FP32 accumulator, issued by one thread.
__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

// Arrive on `mbar` once every MMA issued so far by this thread has completed.
__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// Generic-proxy shared-memory writes become visible to the async proxy (MMA, TMA).
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t holder_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(holder_smem), "r"(ncols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t tmem, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}

// 16 consecutive FP32 columns of this thread's tensor-memory lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// 32 consecutive FP32 columns of this thread's tensor-memory lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// Issue a load of 16 / 32 FP32 columns without waiting; the registers are
// valid after tmem_wait_ld() and reg_fence16/32 on them.
__device__ __forceinline__ void tmem_ld16_async(uint32_t taddr, uint32_t *r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Makes the compiler treat 16 registers as written here, so that no use of a
// tensor-memory load result moves above the preceding tmem_wait_ld().
__device__ __forceinline__ void reg_fence16(uint32_t *r) {
  asm volatile(""
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                 "+r"(r[15]));
}

__device__ __forceinline__ void mbar_arrive(uint32_t addr) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(addr) : "memory");
}

// Barrier among `nthreads` threads (whole warps) of the CTA; id 1..15.
__device__ __forceinline__ void named_sync(uint32_t id, uint32_t nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t addr, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(addr), "r"(count));
}

__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait for the phase with the given parity; false once kWaitLimitNs
// have passed without it completing.
__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity) {
  unsigned long long start = 0;
  for (uint32_t it = 0;; ++it) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred P1;\nmbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2, %3;\n"
        "selp.b32 %0, 1, 0, P1;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity), "r"(kSuspendHintNs)
        : "memory");
    if (done) return true;
    const unsigned long long now = global_ns();
    if (it == 0)
      start = now;
    else if (now - start > kWaitLimitNs)
      return false;
  }
}

// One arrival that also expects `bytes` of asynchronous transactions.
__device__ __forceinline__ void mbar_expect_tx(uint32_t addr, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(addr), "r"(bytes) : "memory");
}

// Bulk copy global -> shared (both 16-byte aligned, bytes a multiple of 16),
// completing `bytes` transactions on `mbar`.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(mbar)
      : "memory");
}

// Bulk copy shared -> global (both 16-byte aligned, bytes a multiple of 16), in
// the current bulk group.
__device__ __forceinline__ void bulk_s2g(void *dst, uint32_t src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(src), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

// Wait until at most N bulk groups still read their shared-memory source.
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}

// Wait until at most N bulk groups are still incomplete.
template <int N>
__device__ __forceinline__ void bulk_wait() {
  asm volatile("cp.async.bulk.wait_group %0;" ::"n"(N) : "memory");
}

// Tiled tensor (TMA) load of one box at coordinates (c0, c1, c2) into shared
// memory, completing its bytes on `mbar`.
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2,
                                            uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(mbar)
      : "memory");
}

// Tiled tensor (TMA) load of one box of a 2D tensor at coordinates (c0, c1).
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int c0, int c1, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
      "[%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(mbar)
      : "memory");
}

// Tiled tensor (TMA) store of one box from shared memory, in the current bulk group.
__device__ __forceinline__ void tma_store_3d(const CUtensorMap *map, int c0, int c1, int c2, uint32_t src) {
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(c0), "r"(c1), "r"(c2), "r"(src)
               : "memory");
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  uint32_t r;
  memcpy(&r, &h, 4);
  return r;
}

// Hardware conversions for the rare inputs of the integer paths below, kept
// out of line so that the common path issues no FP64-pipe instruction.
static __device__ __noinline__ float f64_to_f32_hw(double x) { return __double2float_rn(x); }
static __device__ __noinline__ double f32_to_f64_hw(float f) { return static_cast<double>(f); }

// Integer part of f64_to_f32_rn for results in the FP32 normal range and
// zeros; `ok` is cleared for any other input (then the value is not used).
__device__ __forceinline__ float f64_to_f32_fast(double x, bool &ok) {
  const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(x));
  const uint32_t hi = static_cast<uint32_t>(u >> 32), lo = static_cast<uint32_t>(u);
  const uint32_t e = (hi >> 20) & 0x7FFu;
  const uint32_t m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  const uint32_t rest = lo & 0x1FFFFFFFu;
  uint32_t bits = (hi & 0x80000000u) | ((e - 896u) << 23) | m;
  bits += (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) ? 1u : 0u;
  const bool zero = ((hi & 0x7FFFFFFFu) | lo) == 0u;
  ok = ok && (e - 897u < 254u || zero);
  return __uint_as_float(zero ? (hi & 0x80000000u) : bits);
}

// Integer part of f32_to_f64 for normal numbers and zeros; `ok` is cleared otherwise.
__device__ __forceinline__ double f32_to_f64_fast(float f, bool &ok) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t e = (b >> 23) & 0xFFu;
  const bool zero = (b & 0x7FFFFFFFu) == 0u;
  ok = ok && (e - 1u < 254u || zero);
  const uint32_t hi = zero ? (b & 0x80000000u) : ((b & 0x80000000u) | ((e + 896u) << 20) | ((b & 0x7FFFFFu) >> 3));
  return __hiloint2double(static_cast<int>(hi), zero ? 0 : static_cast<int>(b << 29));
}

// FP64 -> FP32 with round-to-nearest-even (IEEE 754-2008, 4.3.1), by integer
// operations on the bit pattern, so that the conversion does not occupy the
// FP64 pipe (1/64 of the FP32 rate on GB300).  Results in the FP32 normal range
// and zeros take the integer path: the 52-bit significand keeps its top 23 bits
// and is rounded up when the 29 dropped bits exceed half an ulp, or equal it
// with an odd kept part (a carry out of the significand increments the
// exponent, which yields infinity past the largest finite FP32).  Subnormal,
// infinite and NaN results use the hardware conversion.
__device__ __forceinline__ float f64_to_f32_rn(double x) {
  const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(x));
  const uint32_t hi = static_cast<uint32_t>(u >> 32), lo = static_cast<uint32_t>(u);
  const uint32_t e = (hi >> 20) & 0x7FFu;
  const uint32_t sign = hi & 0x80000000u;
  if (e - 897u < 254u) {  // FP32 biased exponent e - 896 in [1, 254]
    const uint32_t m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
    const uint32_t rest = lo & 0x1FFFFFFFu;
    uint32_t bits = sign | ((e - 896u) << 23) | m;
    bits += (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) ? 1u : 0u;
    return __uint_as_float(bits);
  }
  if (((hi & 0x7FFFFFFFu) | lo) == 0u) return __uint_as_float(sign);
  return f64_to_f32_hw(x);
}

// FP32 -> FP64 (exact) by integer operations for normal numbers and zeros:
// exponent rebiased by 1023 - 127, significand shifted left by 29 bits.
// Subnormal, infinite and NaN inputs use the hardware conversion.
__device__ __forceinline__ double f32_to_f64(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t e = (b >> 23) & 0xFFu;
  if (e - 1u < 254u) {
    const uint32_t hi = (b & 0x80000000u) | ((e + 896u) << 20) | ((b & 0x7FFFFFu) >> 3);
    return __hiloint2double(static_cast<int>(hi), static_cast<int>(b << 29));
  }
  if ((b & 0x7FFFFFFFu) == 0u) return __hiloint2double(static_cast<int>(b & 0x80000000u), 0);
  return f32_to_f64_hw(f);
}

// x * 2^s for FP64 x: an integer add to the exponent field when x and the
// result are normal numbers; zeros unchanged; anything else (subnormal,
// infinite, NaN, or a result out of the normal range) by the hardware ldexp.
static __device__ __noinline__ double scale_f64_hw(double x, int s) { return ldexp(x, s); }
__device__ __forceinline__ double scale_f64(double x, int s) {
  const long long u = __double_as_longlong(x);
  const int e = static_cast<int>((u >> 52) & 0x7FF);
  if (e >= 1 && e <= 2046 && e + s >= 1 && e + s <= 2046)
    return __longlong_as_double(u + (static_cast<long long>(s) << 52));
  if ((u & 0x7FFFFFFFFFFFFFFFLL) == 0) return x;
  return scale_f64_hw(x, s);
}

// Binary exponent k of ||F|| (||F|| = f 2^k, f in [0.5, 1)); 0 for a zero or
// non-finite norm.  Double-float images of solution-sized vectors are scaled
// by 2^-k.
__device__ __forceinline__ int df_scale_exp(double nF2) {
  const double nf = sqrt(nF2);
  int k = 0;
  if (nf > 0.0 && isfinite(nf)) frexp(nf, &k);
  return k;
}

// Instruction descriptor of kind::f16 with BF16 A and B, FP32 D, shape M x N;
// b_mn_major = 1 when B is stored MN-major (N contiguous), else K-major.
__host__ __device__ inline uint32_t idesc_bf16(int M, int N, int b_mn_major) {
  uint32_t d = 0;
  d |= 1u << 4;   // D format F32
  d |= 1u << 7;   // A format BF16
  d |= 1u << 10;  // B format BF16
  d |= static_cast<uint32_t>(b_mn_major & 1) << 16;
  d |= static_cast<uint32_t>(N >> 3) << 17;
  d |= static_cast<uint32_t>(M >> 4) << 24;
  return d;
}

// Instruction descriptor of kind::tf32 with TF32 A and B (both K-major), FP32 D.
__host__ __device__ inline uint32_t idesc_tf32(int M, int N) {
  uint32_t d = 0;
  d |= 1u << 4;   // D format F32
  d |= 2u << 7;   // A format TF32
  d |= 2u << 10;  // B format TF32
  d |= static_cast<uint32_t>(N >> 3) << 17;
  d |= static_cast<uint32_t>(M >> 4) << 24;
  return d;
}

// FP32 -> TF32, round to nearest with ties away from zero (cvt.rna), as an
// FP32 value whose low 13 significand bits are zero.
__device__ __forceinline__ float tf32_rna(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return __uint_as_float(r);
}

}  // namespace ptx
}  // namespace stls
