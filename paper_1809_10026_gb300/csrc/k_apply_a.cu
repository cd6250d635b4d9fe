// Fused matrix-free product with the space-time system matrix (Eq. A_kron),
//   A = K_t (x) M_s + M_t (x) J_s + W_t (x) L_s,
// for two and three spatial directions, with the spatial factors expanded by
// direction (Sec. 3):
//   M_s = M_d (x) .. (x) M_1,
//   L_s = sum_k K_k (x) (M elsewhere),
//   J_s = sum_k J_k (x) (M elsewhere) + 2 sum_{k<l} K_k (x) K_l (x) (M elsewhere).
// Three kernels per product, every one streaming its fibers once:
//   slice - directions 1 and 2 of every (b, t[, i_3]) slice, direction 1 through a
//           shared-memory row, direction 2 through a register window;
//   zpass - direction 3 (three spatial directions only);
//   tpass - the time direction, plus W_t (x) L_s on the last time slice
//           (W_t = e e^T with e the last unit vector: only the basis function
//           that is 1 at t = T is non-zero there).
// With the states after directions 1, 2 written as m = M2 M1 x,
// j' = M2 J1 x + J2 M1 x + 2 K2 K1 x and k = M2 K1 x + K2 M1 x, the last spatial
// direction needs M_s x = M3 m, J_s x = M3 j' + J3 m + 2 K3 k, L_s x = M3 k + K3 m:
// 15 banded products per unknown in three spatial directions, each band row
// multiplied once.
#include <cstring>
#include <type_traits>

#include "dot2f.cuh"
#include "kernels.h"
#include "tc_ptx.cuh"

namespace stls {
namespace {

constexpr int kAThreads = 128;

__device__ __forceinline__ void unpack(const float4 &q, float *e) {
  e[0] = q.x;
  e[1] = q.y;
  e[2] = q.z;
  e[3] = q.w;
}
__device__ __forceinline__ void unpack(const double2 &q, double *e) {
  e[0] = q.x;
  e[1] = q.y;
}
__device__ __forceinline__ void unpack(const float4 &q, dfloat *e) {
  e[0].h = q.x;
  e[0].l = q.y;
  e[1].h = q.z;
  e[1].l = q.w;
}
template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
  using V = float4;
};
template <>
struct Vec16<double> {
  using V = double2;
};
template <>
struct Vec16<dfloat> {
  using V = float4;
};

// The W coefficients of one band row, read as whole 16-byte vectors (rows are
// padded to band_row_stride elements).
template <typename T, int W>
__device__ __forceinline__ void load_row(const T *__restrict__ row, T (&c)[W]) {
  using V = typename Vec16<T>::V;
  constexpr int L = 16 / sizeof(T), NV = (W + L - 1) / L;
  const V *v = reinterpret_cast<const V *>(row);
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    T e[L];
    unpack(__ldg(v + k), e);
#pragma unroll
    for (int l = 0; l < L; ++l)
      if (k * L + l < W) c[k * L + l] = e[l];
  }
}

template <typename T, int W>
__device__ __forceinline__ T band_dot(const T (&c)[W], const T (&v)[W], T acc) {
#pragma unroll
  for (int w = 0; w < W; ++w) acc = fma(c[w], v[w], acc);
  return acc;
}

// Double-float form of band_dot: acc + sum_w c_w v_w.  Each product of the
// high parts is split exactly into p + e by one FMA (Dekker's product), p is
// added to the running high sum by Knuth's TwoSum, and e, the TwoSum errors
// and the cross terms c.h v.l + c.l v.h collect in one FP32 low sum; the pair
// is renormalised once at the end (Fast2Sum).  The dropped c.l v.l is below
// 2^-48 of the product.  Explicit _rn operations keep the compiler from
// contracting the error-free transformations into FMAs.
template <int W>
__device__ __forceinline__ dfloat band_dot(const dfloat (&c)[W], const dfloat (&v)[W], dfloat acc) {
  float s = acc.h, lo = acc.l;
#pragma unroll
  for (int w = 0; w < W; ++w) {
    const float p = __fmul_rn(c[w].h, v[w].h);
    float e = __fmaf_rn(c[w].h, v[w].h, -p);
    e = __fmaf_rn(c[w].h, v[w].l, e);
    e = __fmaf_rn(c[w].l, v[w].h, e);
    const float t = __fadd_rn(s, p);
    const float z = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
    lo = __fadd_rn(lo, __fadd_rn(e, err));
    s = t;
  }
  dfloat r;
  r.h = __fadd_rn(s, lo);
  r.l = __fsub_rn(lo, __fsub_rn(r.h, s));
  return r;
}

// a += b in double-float arithmetic (TwoSum of the high parts, then Fast2Sum).
__device__ __forceinline__ dfloat &operator+=(dfloat &a, const dfloat &b) {
  const float t = __fadd_rn(a.h, b.h);
  const float z = __fsub_rn(t, a.h);
  const float err = __fadd_rn(__fsub_rn(a.h, __fsub_rn(t, z)), __fsub_rn(b.h, z));
  const float lo = __fadd_rn(__fadd_rn(a.l, b.l), err);
  a.h = __fadd_rn(t, lo);
  a.l = __fsub_rn(lo, __fsub_rn(a.h, t));
  return a;
}

template <typename T, int W>
__device__ __forceinline__ void slide(T (&win)[W], T v) {
#pragma unroll
  for (int w = 0; w < W - 1; ++w) win[w] = win[w + 1];
  win[W - 1] = v;
}

// Asynchronous copy of one element into shared memory (zero-filled when
// `valid` is false: no global bytes are read then).
template <typename T>
__device__ __forceinline__ void cp_async_elem(T *smem, const T *gmem, bool valid) {
  const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(sa), "l"(gmem), "n"(sizeof(T)),
               "r"(valid ? static_cast<int>(sizeof(T)) : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Rows of asynchronous copies in flight per input.
template <typename T>
constexpr int prefetch_rows() {
  return sizeof(T) == 4 ? 8 : 4;
}

// Coefficients of band row i: the interior copy `in` when i lies in [lo, hi),
// else loaded from the band array (the few boundary rows).
template <typename T, int W>
__device__ __forceinline__ void band_row(const T *__restrict__ band, int i, int wp, int lo, int hi,
                                         const T (&in)[W], T (&c)[W]) {
  if (i >= lo && i < hi) {
#pragma unroll
    for (int w = 0; w < W; ++w) c[w] = in[w];
  } else {
    load_row<T, W>(band + static_cast<size_t>(i) * wp, c);
  }
}

// ---- directions 1 and 2 --------------------------------------------------------------
// Columns are the (slice, i_1) pairs in order; a CTA owns kAThreads consecutive
// columns (one per thread) and walks i_2.  Each row i_2 of the CTA's columns
// (plus P columns of halo on each side) is staged in shared memory by cp.async
// D rows ahead; every thread forms the direction-1 products M1 x, J1 x, K1 x of
// its column from its 2P+1 neighbours, keeps them in windows of 2P+1 rows, and
// emits the direction-2 outputs of the row P behind.  Interior direction-2
// band rows are held in registers.  Neighbours in another slice meet the zero
// coefficients of the band rows outside the matrix; the FP64 product also
// masks them, so that a non-finite entry reaches no other slice (the FP32 and
// double-float products skip the selects: their inputs are finite).
template <typename T, int P>
__device__ __forceinline__ void slice_body(const SliceArgs<T> &a) {
  constexpr int W = 2 * P + 1, D = prefetch_rows<T>(), R = D + 1;
  constexpr int RW = (kAThreads + 2 * P + 3) / 4 * 4;
  constexpr bool MASK = std::is_same<T, double>::value;
  __shared__ __align__(16) T ring[R][RW];
  const int tid = threadIdx.x, n1 = a.n1, n2 = a.n2, wp = a.row_stride;
  const long long area = static_cast<long long>(n1) * n2;
  const long long ncols = a.slices * n1;
  const long long col = static_cast<long long>(blockIdx.x) * kAThreads + tid;
  const bool act = col < ncols;
  const long long s = act ? col / n1 : 0;
  const int x = act ? static_cast<int>(col - s * n1) : 0;
  const long long own = act ? s * area + x : 0;
  const long long own_o = act ? s * a.out_area + x : 0;  // in the (possibly padded) output slices
  unsigned valid = 0;  // bit w: neighbour i_1 = x - P + w lies in the slice
  if (MASK) {
#pragma unroll
    for (int w = 0; w < W; ++w)
      if (act && x - P + w >= 0 && x - P + w < n1) valid |= 1u << w;
  }
  T cM[W], cJ[W], cK[W];
  load_row<T, W>(a.bM1 + static_cast<size_t>(x) * wp, cM);
  load_row<T, W>(a.bJ1 + static_cast<size_t>(x) * wp, cJ);
  load_row<T, W>(a.bK1 + static_cast<size_t>(x) * wp, cK);
  // halo columns: P on each side, loaded by threads 0 .. 2P-1
  long long halo = 0;
  bool has_halo = false;
  int hslot = 0;
  if (tid < 2 * P) {
    const long long c0 = static_cast<long long>(blockIdx.x) * kAThreads;
    const long long hc = tid < P ? c0 - P + tid : c0 + kAThreads + (tid - P);
    hslot = tid < P ? tid : kAThreads + tid;
    if (hc >= 0 && hc < ncols) {
      const long long hs = hc / n1;
      halo = hs * area + (hc - hs * n1);
      has_halo = true;
    }
  }
  // interior direction-2 band rows
  T iM2[W], iJ2[W], i2K2[W], iK2[W];
  const int lo2 = a.lo2, hi2 = a.hi2;
  if (lo2 < hi2) {
    load_row<T, W>(a.bM2 + static_cast<size_t>(lo2) * wp, iM2);
    load_row<T, W>(a.bJ2 + static_cast<size_t>(lo2) * wp, iJ2);
    load_row<T, W>(a.b2K2 + static_cast<size_t>(lo2) * wp, i2K2);
    load_row<T, W>(a.bK2 + static_cast<size_t>(lo2) * wp, iK2);
  } else {
#pragma unroll
    for (int w = 0; w < W; ++w) iM2[w] = iJ2[w] = i2K2[w] = iK2[w] = T(0);
  }
  // this column's input and outputs, advanced one row (n1 values) per step
  const T *xin = a.x + own;
  const T *hin = a.x + halo;
  auto issue = [&](int y, int slot) {
    if (y < n2) {
      T *row = ring[slot];
      cp_async_elem(row + P + tid, xin + static_cast<long long>(y) * n1, act);
      if (tid < 2 * P) cp_async_elem(row + hslot, hin + static_cast<long long>(y) * n1, has_halo);
    }
    cp_async_commit();
  };
#pragma unroll
  for (int e = 0; e < D; ++e) issue(e, e);
  T wm[W], wj[W], wk[W];
#pragma unroll
  for (int w = 0; w < W; ++w) wm[w] = wj[w] = wk[w] = T(0);
  const bool ls_row = a.ls_last != nullptr && act && (s % a.n_t) == a.n_t - 1;
  const bool need_k = a.ls_last == nullptr || ls_row;
  T *om_p = a.out_m + own_o, *oj_p = a.out_j + own_o;
  T *ok_p = a.ls_last == nullptr ? a.out_k + own_o
                                 : (ls_row ? a.ls_last + (s / a.n_t) * area + x : nullptr);
  int slot = 0;  // ring slot of row yy; row yy + D goes to the slot before it
  // one row yy: direction 1 of row yy (from the staged row), then direction 2
  // of row y = yy - P with band rows c2M, c2J, c22K, c2K
  auto row_step = [&](int yy, const T(&c2M)[W], const T(&c2J)[W], const T(&c22K)[W], const T(&c2K)[W]) {
    cp_async_wait<D - 1>();
    __syncthreads();
    T m0 = T(0), j0 = T(0), k0 = T(0);
    if (yy < n2) {
      const T *row = ring[slot] + tid;
      T u[W];
#pragma unroll
      for (int w = 0; w < W; ++w) {
        u[w] = row[w];
        if (MASK && !((valid >> w) & 1u)) u[w] = T(0);
      }
      m0 = band_dot(cM, u, T(0));
      j0 = band_dot(cJ, u, T(0));
      k0 = band_dot(cK, u, T(0));
    }
    issue(yy + D, slot == 0 ? R - 1 : slot - 1);
    slot = slot == R - 1 ? 0 : slot + 1;
    slide(wm, m0);
    slide(wj, j0);
    slide(wk, k0);
    const int y = yy - P;
    if (y >= 0 && act) {
      const T om = band_dot(c2M, wm, T(0));
      T oj = band_dot(c2M, wj, T(0));
      oj = band_dot(c2J, wm, oj);
      oj = band_dot(c22K, wk, oj);
      const long long off = static_cast<long long>(y) * n1;
      om_p[off] = om;
      oj_p[off] = oj;
      if (need_k) {
        T ok = band_dot(c2M, wk, T(0));
        ok = band_dot(c2K, wm, ok);
        ok_p[off] = ok;
      }
    }
  };
  for (int yy0 = 0; yy0 < n2 + P; yy0 += W) {
    if (yy0 - P >= lo2 && yy0 - P + W <= hi2) {
      // a whole group of interior direction-2 rows: the band rows are the registers
#pragma unroll
      for (int u = 0; u < W; ++u) row_step(yy0 + u, iM2, iJ2, i2K2, iK2);
    } else {
      // boundary groups: the band rows are loaded
      auto edge_step = [&](int u) {
        if (yy0 + u < n2 + P) {
          const int y = yy0 + u - P;
          T c2M[W], c2J[W], c22K[W], c2K[W];
          if (y >= 0) {
            band_row<T, W>(a.bM2, y, wp, lo2, hi2, iM2, c2M);
            band_row<T, W>(a.bJ2, y, wp, lo2, hi2, iJ2, c2J);
            band_row<T, W>(a.b2K2, y, wp, lo2, hi2, i2K2, c22K);
            if (need_k) band_row<T, W>(a.bK2, y, wp, lo2, hi2, iK2, c2K);
          }
          row_step(yy0 + u, c2M, c2J, c22K, c2K);
        }
      };
      if constexpr (sizeof(T) == 4) {
        // unrolled: the window slides become register renames
#pragma unroll
        for (int u = 0; u < W; ++u) edge_step(u);
      } else {
        // the 8-byte types keep the loop: their register budget is spent
#pragma unroll 1
        for (int u = 0; u < W; ++u) edge_step(u);
      }
    }
  }
  cp_async_wait<0>();
}

// The FP32 kernel takes the compiler's register choice (four CTAs per SM);
// the FP64 one is held to three CTAs per SM up to degree 3 (its natural count
// allows two, and the FP64 pipe wants the extra warps); the double-float one
// keeps its natural count.
template <typename T, int P>
__global__ void __launch_bounds__(kAThreads) slice_kernel(const __grid_constant__ SliceArgs<T> a) {
  slice_body<T, P>(a);
}
template <int P>
__global__ void __launch_bounds__(kAThreads, P <= 3 ? 3 : 1) slice_kernel_f64(const __grid_constant__ SliceArgs<double> a) {
  slice_body<double, P>(a);
}

// ---- direction 3 ------------------------------------------------------------------------
// One thread per (b, t, i_1, i_2) column, walking i_3 with a register window of
// 2P+1 rows for each of m, j', k, fed by a register queue of the next 2P+1 rows
// (loads issued 2P+1 rows ahead; the loop is unrolled so that every queue slot
// is a fixed register).  Interior band rows are held in registers.
template <typename T, int P>
__global__ void __launch_bounds__(kAThreads) zpass_kernel(const __grid_constant__ ZArgs<T> a) {
  constexpr int W = 2 * P + 1;
  const int tid = threadIdx.x;
  const long long col = static_cast<long long>(blockIdx.x) * kAThreads + tid;
  if (col >= a.outer * a.inner) return;  // no block-wide barrier below
  const long long inner = a.inner, o = col / inner, cc = col - o * inner;
  const int n = a.n, wp = a.row_stride, lo = a.lo, hi = a.hi;
  const long long base = o * n * inner + cc;
  const T *__restrict__ Im = a.m + base;
  const T *__restrict__ Ij = a.j + base;
  const T *__restrict__ Ik = a.k + base;
  auto ld = [&](const T *__restrict__ p, int r) -> T { return (r >= 0 && r < n) ? p[r * inner] : T(0); };
  T iM[W], iJ[W], i2K[W], iK[W];
  if (lo < hi) {
    load_row<T, W>(a.bM + static_cast<size_t>(lo) * wp, iM);
    load_row<T, W>(a.bJ + static_cast<size_t>(lo) * wp, iJ);
    load_row<T, W>(a.b2K + static_cast<size_t>(lo) * wp, i2K);
    load_row<T, W>(a.bK + static_cast<size_t>(lo) * wp, iK);
  } else {
#pragma unroll
    for (int w = 0; w < W; ++w) iM[w] = iJ[w] = i2K[w] = iK[w] = T(0);
  }
  T wm[W], wj[W], wk[W], qm[W], qj[W], qk[W];
#pragma unroll
  for (int w = 0; w < W; ++w) {
    wm[w] = ld(Im, w - P);
    wj[w] = ld(Ij, w - P);
    wk[w] = ld(Ik, w - P);
    qm[w] = ld(Im, P + 1 + w);
    qj[w] = ld(Ij, P + 1 + w);
    qk[w] = ld(Ik, P + 1 + w);
  }
  const bool ls_col = a.ls_last != nullptr && (o % a.n_t) == a.n_t - 1;
  T *ls = ls_col ? a.ls_last + (o / a.n_t) * n * inner + cc : nullptr;
  // outputs of row i from the window, with band rows cM, cJ, c2K, cK
  auto emit = [&](int i, const T(&cM)[W], const T(&cJ)[W], const T(&c2K)[W], const T(&cK)[W]) {
    const T oms = band_dot(cM, wm, T(0));
    T ojs = band_dot(cM, wj, T(0));
    ojs = band_dot(cJ, wm, ojs);
    ojs = band_dot(c2K, wk, ojs);
    a.Ms[base + static_cast<long long>(i) * inner] = oms;
    a.Js[base + static_cast<long long>(i) * inner] = ojs;
    if (ls_col) ls[static_cast<long long>(i) * inner] = band_dot(cK, wm, band_dot(cM, wk, T(0)));
  };
  // the window takes row i + P + 1 from queue slot u, which then loads row i + P + 1 + W
  auto advance = [&](int i, int u) {
    slide(wm, qm[u]);
    slide(wj, qj[u]);
    slide(wk, qk[u]);
    qm[u] = ld(Im, i + P + 1 + W);
    qj[u] = ld(Ij, i + P + 1 + W);
    qk[u] = ld(Ik, i + P + 1 + W);
  };
  for (int i0 = 0; i0 < n; i0 += W) {
    if (i0 >= lo && i0 + W <= hi) {
      // a whole group of interior rows: the band rows are the registers
#pragma unroll
      for (int u = 0; u < W; ++u) {
        emit(i0 + u, iM, iJ, i2K, iK);
        advance(i0 + u, u);
      }
    } else {
#pragma unroll
      for (int u = 0; u < W; ++u) {
        const int i = i0 + u;
        if (i < n) {
          T cM[W], cJ[W], c2K[W], cK[W];
          band_row<T, W>(a.bM, i, wp, lo, hi, iM, cM);
          band_row<T, W>(a.bJ, i, wp, lo, hi, iJ, cJ);
          band_row<T, W>(a.b2K, i, wp, lo, hi, i2K, c2K);
          if (ls_col) band_row<T, W>(a.bK, i, wp, lo, hi, iK, cK);
          emit(i, cM, cJ, c2K, cK);
        }
        advance(i, u);
      }
    }
  }
}

// ---- time direction -------------------------------------------------------------------
// y = K_t (x) (M_s x) + M_t (x) (J_s x), and + L_s x on the last time slice;
// same register window and queue as the direction-3 pass.  Grid: x over the
// N_s columns, y over the right-hand sides.  With FUSE (FP32) every thread
// also accumulates (p, y) over its column, and the blocks of a right-hand side
// combine their sums in a fixed order; the last one sets alpha.
template <typename T, int P, bool FUSE>
__global__ void __launch_bounds__(kAThreads) tpass_kernel(const __grid_constant__ TArgs<T> a) {
  constexpr int W = 2 * P + 1;
  const int tid = threadIdx.x;
  const long long inner = a.inner, o = blockIdx.y;
  const long long cc = static_cast<long long>(blockIdx.x) * kAThreads + tid;
  Dot2f acc;
  if (cc < inner) {
    const int n = a.n, wp = a.row_stride, lo = a.lo, hi = a.hi;
    const long long base = o * n * inner + cc;
    const T *__restrict__ Ims = a.Ms + base;
    const T *__restrict__ Ijs = a.Js + base;
    auto ld = [&](const T *__restrict__ p, int r) -> T { return (r >= 0 && r < n) ? p[r * inner] : T(0); };
    T iK[W], iM[W];
    if (lo < hi) {
      load_row<T, W>(a.bK + static_cast<size_t>(lo) * wp, iK);
      load_row<T, W>(a.bM + static_cast<size_t>(lo) * wp, iM);
    } else {
#pragma unroll
      for (int w = 0; w < W; ++w) iK[w] = iM[w] = T(0);
    }
    T wm[W], wj[W], qm[W], qj[W];
    float qp[W];  // FUSE: p of rows i0 + u, loaded W rows ahead
    const float *Ip = nullptr;
    if constexpr (FUSE) Ip = a.fuse.p + base;
    auto ldp = [&](int r) -> float {
      if constexpr (FUSE)
        return r < n ? Ip[r * inner] : 0.f;
      else
        return 0.f;
    };
#pragma unroll
    for (int w = 0; w < W; ++w) {
      wm[w] = ld(Ims, w - P);
      wj[w] = ld(Ijs, w - P);
      qm[w] = ld(Ims, P + 1 + w);
      qj[w] = ld(Ijs, P + 1 + w);
      qp[w] = ldp(w);
    }
    auto emit = [&](int i, int u, const T(&cK)[W], const T(&cM)[W]) {
      T out = band_dot(cK, wm, T(0));
      out = band_dot(cM, wj, out);
      if (i == n - 1) out += a.ls_last[o * inner + cc];
      a.y[base + static_cast<long long>(i) * inner] = out;
      if constexpr (FUSE) acc.add(qp[u], out);
    };
    auto advance = [&](int i, int u) {
      slide(wm, qm[u]);
      slide(wj, qj[u]);
      qm[u] = ld(Ims, i + P + 1 + W);
      qj[u] = ld(Ijs, i + P + 1 + W);
      if constexpr (FUSE) qp[u] = ldp(i + W);
    };
    for (int i0 = 0; i0 < n; i0 += W) {
      if (i0 >= lo && i0 + W <= hi) {
#pragma unroll
        for (int u = 0; u < W; ++u) {
          emit(i0 + u, u, iK, iM);
          advance(i0 + u, u);
        }
      } else {
#pragma unroll
        for (int u = 0; u < W; ++u) {
          const int i = i0 + u;
          if (i < n) {
            T cK[W], cM[W];
            band_row<T, W>(a.bK, i, wp, lo, hi, iK, cK);
            band_row<T, W>(a.bM, i, wp, lo, hi, iM, cM);
            emit(i, u, cK, cM);
          }
          advance(i, u);
        }
      }
    }
  }  // cc < inner
  if constexpr (FUSE) {
    // block sum in a fixed order, then the blocks of this right-hand side
    __shared__ double sh[kAThreads / 32];
    __shared__ bool is_last;
    const int lane = tid & 31, wid = tid >> 5;
    double v = acc.value();
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    const unsigned gx = gridDim.x;
    const AlphaFuse &fz = a.fuse;
    if (tid == 0) {
      double t = 0.0;
#pragma unroll
      for (int w = 0; w < kAThreads / 32; ++w) t += sh[w];
      fz.partials[o * gx + blockIdx.x] = t;
      __threadfence();
      is_last = atomicAdd(fz.tickets + o, 1u) == gx - 1;
    }
    __syncthreads();
    if (is_last) {
      __threadfence();
      const volatile double *src = fz.partials + o * gx;
      double t = 0.0;
      for (unsigned g = tid; g < gx; g += kAThreads) t += src[g];
#pragma unroll
      for (int s = 16; s > 0; s >>= 1) t += __shfl_xor_sync(0xffffffffu, t, s);
      __syncthreads();
      if (lane == 0) sh[wid] = t;
      __syncthreads();
      if (tid == 0) {
        double tot = 0.0;
#pragma unroll
        for (int w = 0; w < kAThreads / 32; ++w) tot += sh[w];
        fz.tickets[o] = 0u;
        CGState &st = fz.st[o];
        if (st.active) {
          st.pq = tot;
          if (!isfinite(tot)) {
            st.status = STLS_ENONFINITE;
            st.active = 0;
          } else if (!(tot > 0.0)) {
            st.status = STLS_EBREAKDOWN;
            st.active = 0;
          } else {
            st.alpha = st.rz / tot;
          }
        }
      }
    }
  }
}

// ---- direction 3 and time in one sweep (FP32) -----------------------------------------
// A CTA owns 32 consecutive columns c = (i_1, i_2) (one warp per i_3 row, so
// every access is a 128-byte row segment), Z consecutive rows i_3 and one
// right-hand side; thread (i_3, c) walks t.  At each t the CTA stages the rows
// i_3 = z0 - P .. z0 + Z + P - 1 of m, j', k in shared memory (16-byte
// cp.async, D time slices ahead; rows outside the mesh are zero-filled): the
// direction-1/2 kernel writes these three states with every (t, i_3) slice
// padded to a multiple of 4 values, so that row segments are 16-byte aligned.
// Each thread forms
//   M_s x = M3 m,  J_s x = M3 j' + J3 m + 2 K3 k   (and L_s x = M3 k + K3 m on
//   the last time slice)
// from 2P+1 staged rows, keeps M_s x and J_s x in time windows of 2P+1 rows and
// emits y = K_t (M_s x) + M_t (J_s x) (+ L_s x on the last slice) for the time
// row P behind: 4 vector passes instead of the 8 of a direction-3 pass and a
// time pass (5 with the fused (p, A p)).  Each sum of several band products is
// formed as independent FMA chains, one per band, added at the end; two chains
// over the same band length run as one chain of paired FP32 FMAs (__ffma2_rn:
// M3 m with M3 j', and K_t (M_s x) with M_t (J_s x) from a window of pairs),
// which halves their instructions and rounds like two separate chains.  The band
// rows shared by the interior rows of direction 3 and of time are kernel
// parameters (constant bank); warps of a boundary row i_3 read theirs from
// the band arrays, and time groups touching a boundary row or the last slice
// take a checked path.
constexpr int kZtCols = 32;
constexpr int kZtDepth = 4;
constexpr int kZtMaxZ = 12;
constexpr int kZtChunks = 2;  // 16-byte chunks a thread stages per time slice (checked on the host)
constexpr int kZtMaxW = 2 * kFusedMaxP + 1;

struct ZTArgs {
  const float *m, *j, *k;  // (b, t, i_3) slices of `pitch` values (n1 n2 rounded up to 4)
  float *y;
  AlphaFuse fuse;
  const float *bM3, *bJ3, *bK3, *b2K3;  // padded direction-3 bands (row stride ws)
  const float *bKt, *bMt;               // padded time bands (row stride wt)
  float2 iKM[kZtMaxW];                  // (K_t, M_t) of the time band rows [lo_t, hi_t), all equal
  float i3[4][kZtMaxW];                 // rows [lo3, hi3) of M3, J3, 2 K3, K3 all equal these
  float2 i3mm[kZtMaxW];                 // (M3, M3) of that row, for paired products
  long long inner, pitch;               // n1 n2 and its rounding up to a multiple of 4
  int n3, nt, Z, ws, wt, lo3, hi3, lo_t, hi_t;
};

// 16-byte asynchronous copy into shared memory (zero-filled when `valid` is
// false: no global bytes are read then).
__device__ __forceinline__ void cp_async16(float *smem, const float *gmem, bool valid) {
  const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(valid ? 16 : 0)
               : "memory");
}

template <int W>
__device__ __forceinline__ float chain_g(const float *__restrict__ c, const float (&v)[W]) {  // c in global memory
  float acc = 0.f;
#pragma unroll
  for (int w = 0; w < W; ++w) acc = fmaf(__ldg(c + w), v[w], acc);
  return acc;
}

template <int P, bool FUSE>
__global__ void __launch_bounds__(kZtCols * kZtMaxZ, 2) zt_kernel(const __grid_constant__ ZTArgs a) {
  constexpr int W = 2 * P + 1, D = kZtDepth, R = D + 1, KC = kZtChunks;
  extern __shared__ __align__(16) float zt_smem[];
  const int tx = threadIdx.x, ty = threadIdx.y, Z = a.Z, ZR = Z + 2 * P;
  const int tid = ty * kZtCols + tx, nth = Z * kZtCols;
  const int n3 = a.n3, nt = a.nt;
  const long long inner = a.inner, slice = static_cast<long long>(n3) * inner;
  const long long pslice = static_cast<long long>(n3) * a.pitch;
  const long long c0 = static_cast<long long>(blockIdx.x) * kZtCols, cc = c0 + tx;
  const int z0 = blockIdx.y * Z, i3 = z0 + ty;
  const bool act = cc < inner && i3 < n3;
  const bool bdry = i3 < n3 && (i3 < a.lo3 || i3 >= a.hi3);  // the same in the whole warp
  const long long b = blockIdx.z;
  // y and p of (b, t = 0, i_3, c) in the natural order
  const long long obase = b * nt * slice + static_cast<long long>(i3 < n3 ? i3 : 0) * inner + (cc < inner ? cc : 0);
  const int roff = (i3 < n3 ? i3 : 0) * a.ws;  // this row of the direction-3 bands
  // this thread's 16-byte chunks of a staged slice: chunk e = tid + q nth of
  // the 3 x ZR x 8 chunks (array, row, 4 columns)
  // slot: m, j', k rows, then (FUSE) p of this CTA's (i_3, c) at time t - P
  const int arr_floats = ZR * kZtCols, slot_floats = 3 * arr_floats + (FUSE ? Z * kZtCols : 0);
  const float *gsrc[KC];
  int sdst[KC];
  unsigned vmask = 0, nk = 0;
#pragma unroll
  for (int q = 0; q < KC; ++q) {
    const int e = tid + q * nth;
    gsrc[q] = a.m;
    sdst[q] = 0;
    if (e < 3 * ZR * 8) {
      nk = q + 1;
      const int arr = e / (ZR * 8), rem = e - arr * (ZR * 8), row = rem >> 3, ch = rem & 7;
      const int gi3 = z0 - P + row;
      const long long col = c0 + 4 * ch;
      const float *base = arr == 0 ? a.m : (arr == 1 ? a.j : a.k);
      sdst[q] = arr * arr_floats + row * kZtCols + 4 * ch;
      gsrc[q] = base + b * nt * pslice;
      if (gi3 >= 0 && gi3 < n3 && col < a.pitch) {
        gsrc[q] += static_cast<long long>(gi3) * a.pitch + col;
        vmask |= 1u << q;
      }
    }
  }
  auto issue = [&](int t, int slot) {
    if (t < nt) {
      const long long toff = static_cast<long long>(t) * pslice;
      float *dst = zt_smem + slot * slot_floats;
#pragma unroll
      for (int q = 0; q < KC; ++q)
        if (q < static_cast<int>(nk)) cp_async16(dst + sdst[q], gsrc[q] + toff, (vmask >> q) & 1u);
      if constexpr (FUSE)
        if (t >= P) cp_async_elem(dst + 3 * arr_floats + tid, a.fuse.p + obase + static_cast<long long>(t - P) * slice, act);
    }
    cp_async_commit();
  };
#pragma unroll
  for (int e = 0; e < D; ++e) issue(e, e);
  float2 win[W];  // time window of (M_s x, J_s x): one paired FMA per band term
#pragma unroll
  for (int w = 0; w < W; ++w) win[w] = make_float2(0.f, 0.f);
  float ls = 0.f;  // L_s x of the last time slice
  Dot2f acc;
  int slot = 0;
  // time row tt: M_s x and J_s x from the staged rows into the windows, then
  // y of time row tt - P.  FAST: tt < nt - 1 and row tt - P an interior time row.
  auto step = [&](int tt, auto fast) {
    constexpr bool FAST = decltype(fast)::value;
    const int y = tt - P;
    const bool emit = FAST || (y >= 0 && y < nt);
    [[maybe_unused]] float pv = 0.f;  // p of the emitted row: staged with the slice, or loaded in the last P steps
    if constexpr (FUSE)
      if (!FAST && tt >= nt && emit && act) pv = a.fuse.p[obase + static_cast<long long>(y) * slice];
    float ms = 0.f, js = 0.f;
    if (FAST || tt < nt) {
      cp_async_wait<D - 1>();
      __syncthreads();
      if constexpr (FUSE)
        if (emit) pv = zt_smem[slot * slot_floats + 3 * arr_floats + tid];
      const float *sm = zt_smem + slot * slot_floats + ty * kZtCols + tx;
      float mv[W], jv[W], kv[W];
#pragma unroll
      for (int w = 0; w < W; ++w) {
        mv[w] = sm[w * kZtCols];
        jv[w] = sm[arr_floats + w * kZtCols];
        kv[w] = sm[2 * arr_floats + w * kZtCols];
      }
      if (!bdry) {
        // M3 m and M3 j' as the two halves of one paired FMA chain
        float2 mj = make_float2(0.f, 0.f);
        float j2 = 0.f, j3 = 0.f;
#pragma unroll
        for (int w = 0; w < W; ++w) {
          mj = __ffma2_rn(a.i3mm[w], make_float2(mv[w], jv[w]), mj);
          j2 = fmaf(a.i3[1][w], mv[w], j2);
          j3 = fmaf(a.i3[2][w], kv[w], j3);
        }
        ms = mj.x;
        js = (mj.y + j2) + j3;
        if (!FAST && tt == nt - 1) {
          float l1 = 0.f, l2 = 0.f;
#pragma unroll
          for (int w = 0; w < W; ++w) {
            l1 = fmaf(a.i3[0][w], kv[w], l1);
            l2 = fmaf(a.i3[3][w], mv[w], l2);
          }
          ls = l1 + l2;
        }
      } else {
        ms = chain_g(a.bM3 + roff, mv);
        js = (chain_g(a.bM3 + roff, jv) + chain_g(a.bJ3 + roff, mv)) + chain_g(a.b2K3 + roff, kv);
        if (!FAST && tt == nt - 1) ls = chain_g(a.bM3 + roff, kv) + chain_g(a.bK3 + roff, mv);
      }
      issue(tt + D, slot == 0 ? R - 1 : slot - 1);
      slot = slot == R - 1 ? 0 : slot + 1;
    }
    slide(win, make_float2(ms, js));
    if (emit) {
      // K_t (M_s x) and M_t (J_s x) as the two halves of one paired FMA chain
      float2 o = make_float2(0.f, 0.f);
      if (FAST || (y >= a.lo_t && y < a.hi_t)) {
#pragma unroll
        for (int w = 0; w < W; ++w) o = __ffma2_rn(a.iKM[w], win[w], o);
      } else {
        const float *rK = a.bKt + static_cast<size_t>(y) * a.wt, *rM = a.bMt + static_cast<size_t>(y) * a.wt;
#pragma unroll
        for (int w = 0; w < W; ++w) o = __ffma2_rn(make_float2(__ldg(rK + w), __ldg(rM + w)), win[w], o);
      }
      float out = o.x + o.y;
      if (!FAST && y == nt - 1) out += ls;
      if (act) {
        a.y[obase + static_cast<long long>(y) * slice] = out;
        if constexpr (FUSE) acc.add(pv, out);
      }
    }
  };
  for (int t0 = 0; t0 < nt + P; t0 += W) {
    if (t0 - P >= a.lo_t && t0 - P + W <= a.hi_t && t0 + W <= nt - 1) {
#pragma unroll
      for (int u = 0; u < W; ++u) step(t0 + u, std::true_type{});
    } else {
#pragma unroll
      for (int u = 0; u < W; ++u)
        if (t0 + u < nt + P) step(t0 + u, std::false_type{});
    }
  }
  cp_async_wait<0>();
  if constexpr (FUSE) {
    // block sum in a fixed order, then the blocks of this right-hand side
    __shared__ double sh[kZtMaxZ];
    __shared__ bool is_last;
    double v = acc.value();
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
    if (tx == 0) sh[ty] = v;
    __syncthreads();
    const unsigned nb = gridDim.x * gridDim.y, bi = blockIdx.y * gridDim.x + blockIdx.x, o = blockIdx.z;
    const AlphaFuse &fz = a.fuse;
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < Z; ++w) t += sh[w];
      fz.partials[static_cast<size_t>(o) * nb + bi] = t;
      __threadfence();
      is_last = atomicAdd(fz.tickets + o, 1u) == nb - 1;
    }
    __syncthreads();
    if (is_last) {
      __threadfence();
      const volatile double *src = fz.partials + static_cast<size_t>(o) * nb;
      double t = 0.0;
      for (unsigned g = tid; g < nb; g += nth) t += src[g];
#pragma unroll
      for (int s = 16; s > 0; s >>= 1) t += __shfl_xor_sync(0xffffffffu, t, s);
      __syncthreads();
      if (tx == 0) sh[ty] = t;
      __syncthreads();
      if (tid == 0) {
        double tot = 0.0;
        for (int w = 0; w < Z; ++w) tot += sh[w];
        fz.tickets[o] = 0u;
        CGState &st = fz.st[o];
        if (st.active) {
          st.pq = tot;
          if (!isfinite(tot)) {
            st.status = STLS_ENONFINITE;
            st.active = 0;
          } else if (!(tot > 0.0)) {
            st.status = STLS_EBREAKDOWN;
            st.active = 0;
          } else {
            st.alpha = st.rz / tot;
          }
        }
      }
    }
  }
}

// ---- double-float images of FP64 vectors ------------------------------------------------
constexpr int kDfThreads = 256;

__global__ void __launch_bounds__(kDfThreads)
    df_split_kernel(const double *__restrict__ x, dfloat *__restrict__ y, long long N, const CGState *scale) {
  const int b = blockIdx.y;
  const int k = scale != nullptr ? ptx::df_scale_exp(scale[b].nF2) : 0;
  const double *xb = x + static_cast<size_t>(b) * N;
  dfloat *yb = y + static_cast<size_t>(b) * N;
  for (long long i = blockIdx.x * static_cast<long long>(kDfThreads) + threadIdx.x; i < N;
       i += static_cast<long long>(gridDim.x) * kDfThreads) {
    const double v = ptx::scale_f64(xb[i], -k);
    dfloat o;
    o.h = ptx::f64_to_f32_rn(v);
    o.l = ptx::f64_to_f32_rn(v - ptx::f32_to_f64(o.h));  // v - h is exact in FP64
    yb[i] = o;
  }
}

__global__ void __launch_bounds__(kDfThreads)
    df_join_kernel(const dfloat *__restrict__ y, double *__restrict__ x, long long N, const CGState *scale) {
  const int b = blockIdx.y;
  const int k = scale != nullptr ? ptx::df_scale_exp(scale[b].nF2) : 0;
  const dfloat *yb = y + static_cast<size_t>(b) * N;
  double *xb = x + static_cast<size_t>(b) * N;
  for (long long i = blockIdx.x * static_cast<long long>(kDfThreads) + threadIdx.x; i < N;
       i += static_cast<long long>(gridDim.x) * kDfThreads) {
    const dfloat o = yb[i];
    xb[i] = ptx::scale_f64(ptx::f32_to_f64(o.h) + ptx::f32_to_f64(o.l), k);
  }
}

unsigned df_grid(long long N) {
  const long long g = (N + kDfThreads - 1) / kDfThreads;
  return static_cast<unsigned>(g < 1 ? 1 : (g > 152 * 16 ? 152 * 16 : g));
}

long long blocks_for(long long cols) { return (cols + kAThreads - 1) / kAThreads; }

template <typename T, int P>
cudaError_t launch_slice_p(const SliceArgs<T> &a, cudaStream_t s) {
  const long long g = (a.slices * a.n1 + kAThreads - 1) / kAThreads;
  if (g > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  if (g > 0) {
    if constexpr (std::is_same<T, double>::value)
      slice_kernel_f64<P><<<static_cast<unsigned>(g), kAThreads, 0, s>>>(a);
    else
      slice_kernel<T, P><<<static_cast<unsigned>(g), kAThreads, 0, s>>>(a);
  }
  return cudaGetLastError();
}
template <typename T, int P>
cudaError_t launch_zpass_p(const ZArgs<T> &a, cudaStream_t s) {
  const long long g = blocks_for(a.outer * a.inner);
  if (g > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  if (g > 0) zpass_kernel<T, P><<<static_cast<unsigned>(g), kAThreads, 0, s>>>(a);
  return cudaGetLastError();
}
template <typename T, int P>
cudaError_t launch_tpass_p(const TArgs<T> &a, cudaStream_t s) {
  const long long g = blocks_for(a.inner);
  if (g > 0x7fffffffLL || a.outer > 65535) return cudaErrorInvalidConfiguration;
  if (g > 0 && a.outer > 0) {
    const dim3 grid(static_cast<unsigned>(g), static_cast<unsigned>(a.outer));
    if constexpr (std::is_same<T, float>::value) {
      if (a.fuse.p != nullptr) {
        tpass_kernel<T, P, true><<<grid, kAThreads, 0, s>>>(a);
        return cudaGetLastError();
      }
    }
    tpass_kernel<T, P, false><<<grid, kAThreads, 0, s>>>(a);
  }
  return cudaGetLastError();
}

// Rows of i_3 per CTA of the fused direction-3 and time kernel: n3 split into
// ceil(n3 / 12) equal groups (65 -> 6 x 11); 0 when n3 < 8 (the two passes
// are used then).
int zt_rows(int n3, int p) {
  if (n3 < 8) return 0;
  const int groups = (n3 + kZtMaxZ - 1) / kZtMaxZ;
  const int Z = (n3 + groups - 1) / groups;
  // every thread stages at most kZtChunks 16-byte chunks of the 3 (Z + 2p) rows
  return 3 * (Z + 2 * p) * 8 <= kZtChunks * kZtCols * Z ? Z : 0;
}

template <int P>
cudaError_t launch_zt_p(const ZTArgs &a, int B, cudaStream_t s) {
  const long long gx = (a.inner + kZtCols - 1) / kZtCols;
  const int gy = (a.n3 + a.Z - 1) / a.Z;
  if (gx > 0x7fffffffLL || B > 65535) return cudaErrorInvalidConfiguration;
  const bool fuse = a.fuse.p != nullptr;
  const size_t smem = static_cast<size_t>(kZtDepth + 1) * (3 * (a.Z + 2 * P) + (fuse ? a.Z : 0)) * kZtCols *
                      sizeof(float);
  static size_t raised[2] = {0, 0};  // dynamic shared memory already allowed, per variant
  if (smem > 48 * 1024 && raised[fuse] < smem) {
    cudaError_t e = fuse ? cudaFuncSetAttribute(zt_kernel<P, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                static_cast<int>(smem))
                         : cudaFuncSetAttribute(zt_kernel<P, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    raised[fuse] = smem;
  }
  if (gx > 0 && B > 0) {
    const dim3 grid(static_cast<unsigned>(gx), static_cast<unsigned>(gy), static_cast<unsigned>(B));
    const dim3 block(kZtCols, static_cast<unsigned>(a.Z));
    if (fuse)
      zt_kernel<P, true><<<grid, block, smem, s>>>(a);
    else
      zt_kernel<P, false><<<grid, block, smem, s>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t dispatch_zt(int p, const ZTArgs &a, int B, cudaStream_t s) {
  switch (p) {
    case 1: return launch_zt_p<1>(a, B, s);
    case 2: return launch_zt_p<2>(a, B, s);
    case 3: return launch_zt_p<3>(a, B, s);
    case 4: return launch_zt_p<4>(a, B, s);
    default: return cudaErrorInvalidValue;  // degrees 5, 6 take the two passes
  }
}

template <typename T>
cudaError_t dispatch_slice(int p, const SliceArgs<T> &a, cudaStream_t s) {
  switch (p) {
    case 1: return launch_slice_p<T, 1>(a, s);
    case 2: return launch_slice_p<T, 2>(a, s);
    case 3: return launch_slice_p<T, 3>(a, s);
    case 4: return launch_slice_p<T, 4>(a, s);
    case 5: return launch_slice_p<T, 5>(a, s);
    case 6: return launch_slice_p<T, 6>(a, s);
    default: return cudaErrorInvalidValue;
  }
}
template <typename T>
cudaError_t dispatch_zpass(int p, const ZArgs<T> &a, cudaStream_t s) {
  switch (p) {
    case 1: return launch_zpass_p<T, 1>(a, s);
    case 2: return launch_zpass_p<T, 2>(a, s);
    case 3: return launch_zpass_p<T, 3>(a, s);
    case 4: return launch_zpass_p<T, 4>(a, s);
    case 5: return launch_zpass_p<T, 5>(a, s);
    case 6: return launch_zpass_p<T, 6>(a, s);
    default: return cudaErrorInvalidValue;
  }
}
template <typename T>
cudaError_t dispatch_tpass(int p, const TArgs<T> &a, cudaStream_t s) {
  switch (p) {
    case 1: return launch_tpass_p<T, 1>(a, s);
    case 2: return launch_tpass_p<T, 2>(a, s);
    case 3: return launch_tpass_p<T, 3>(a, s);
    case 4: return launch_tpass_p<T, 4>(a, s);
    case 5: return launch_tpass_p<T, 5>(a, s);
    case 6: return launch_tpass_p<T, 6>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

// Partial sums of the fused (p, A p): one per block of the last kernel of the
// product, at most ceil(N_s / 128) (time pass) or ceil(n1 n2 / 32) ceil(n3 / Z)
// <= N_s / 32 + 129 (fused direction-3 and time kernel, Z >= 8, n3 <= 128).
int alpha_blocks(long long Ns) { return static_cast<int>(4 * blocks_for(Ns) + 129); }

int band_row_stride(int p, int elem_bytes) {
  const int w = 2 * p + 1, l = 16 / elem_bytes;
  return (w + l - 1) / l * l;
}

bool fused_A_supported(int d, int p_s, int p_t) {
  return (d == 2 || d == 3) && p_s >= 1 && p_s <= kFusedMaxP && p_t >= 1 && p_t <= kFusedMaxP;
}

template <typename T>
cudaError_t launch_fused_A(const FusedA<T> &f, const T *x, T *y, cudaStream_t s) {
  if (!fused_A_supported(f.d, f.p_s, f.p_t) || f.B < 1 || f.n_t < 1) return cudaErrorInvalidValue;
  for (int k = 0; k < f.d; ++k)
    if (f.n[k] < 1 || f.n[k] > 128) return cudaErrorInvalidValue;
  const long long n1 = f.n[0], n2 = f.n[1], n3 = f.d == 3 ? f.n[2] : 1;
  const long long Ns = n1 * n2 * n3;
  const int ws = band_row_stride(f.p_s, sizeof(T)), wt = band_row_stride(f.p_t, sizeof(T));
  // directions 1, 2
  SliceArgs<T> sa{};
  sa.x = x;
  sa.bM1 = f.bM[0];
  sa.bJ1 = f.bJ[0];
  sa.bK1 = f.bK[0];
  sa.bM2 = f.bM[1];
  sa.bJ2 = f.bJ[1];
  sa.bK2 = f.bK[1];
  sa.b2K2 = f.b2K[1];
  sa.slices = static_cast<long long>(f.B) * f.n_t * n3;
  // FP32, three spatial directions: direction 3 and time in one kernel, which
  // reads m, j', k in slices padded to 16 bytes
  int zt_Z = 0;
  if constexpr (std::is_same<T, float>::value)
    // degrees 5, 6: the two passes (the fused kernel spills at two CTAs per SM and
    // is slower than the passes at one)
    if (f.d == 3 && f.p_t == f.p_s && f.p_s <= 4) zt_Z = zt_rows(f.n[2], f.p_s);
  const long long pitch = zt_Z > 0 ? (n1 * n2 + 3) / 4 * 4 : n1 * n2;
  sa.out_area = pitch;
  sa.n1 = f.n[0];
  sa.n2 = f.n[1];
  sa.n_t = f.n_t;
  sa.row_stride = ws;
  sa.lo2 = f.lo[1];
  sa.hi2 = f.hi[1];
  T *Ms = f.work[3], *Js = f.work[4];
  if (f.d == 3) {
    sa.out_m = f.work[0];
    sa.out_j = f.work[1];
    sa.out_k = f.work[2];
    sa.ls_last = nullptr;
  } else {
    sa.out_m = Ms;
    sa.out_j = Js;
    sa.out_k = nullptr;
    sa.ls_last = f.ls_last;
  }
  cudaError_t e = dispatch_slice<T>(f.p_s, sa, s);
  if (e != cudaSuccess) return e;
  if constexpr (std::is_same<T, float>::value) {
    if (zt_Z > 0) {
      ZTArgs za{};
      za.m = f.work[0];
      za.j = f.work[1];
      za.k = f.work[2];
      za.y = y;
      za.fuse = f.fuse;
      za.bM3 = f.bM[2];
      za.bJ3 = f.bJ[2];
      za.bK3 = f.bK[2];
      za.b2K3 = f.b2K[2];
      za.bKt = f.bKt;
      za.bMt = f.bMt;
      za.inner = n1 * n2;
      za.pitch = pitch;
      za.n3 = f.n[2];
      za.nt = f.n_t;
      za.Z = zt_Z;
      za.ws = ws;
      za.wt = wt;
      za.lo_t = f.lo_t;
      za.hi_t = f.hi_t;
      za.lo3 = f.lo[2];
      za.hi3 = f.hi[2];
      for (int r = 0; r < 4; ++r)
        for (int w = 0; w < 2 * f.p_s + 1; ++w) za.i3[r][w] = f.lo[2] < f.hi[2] ? f.i3[r][w] : 0.f;
      for (int w = 0; w < 2 * f.p_s + 1; ++w) za.i3mm[w] = make_float2(za.i3[0][w], za.i3[0][w]);
      for (int w = 0; w < 2 * f.p_t + 1; ++w) {
        za.iKM[w] = f.lo_t < f.hi_t ? make_float2(f.iKt[w], f.iMt[w]) : make_float2(0.f, 0.f);
      }
      return dispatch_zt(f.p_s, za, f.B, s);
    }
  }
  // direction 3
  if (f.d == 3) {
    ZArgs<T> za{};
    za.m = f.work[0];
    za.j = f.work[1];
    za.k = f.work[2];
    za.Ms = Ms;
    za.Js = Js;
    za.ls_last = f.ls_last;
    za.bM = f.bM[2];
    za.bJ = f.bJ[2];
    za.bK = f.bK[2];
    za.b2K = f.b2K[2];
    za.outer = static_cast<long long>(f.B) * f.n_t;
    za.inner = n1 * n2;
    za.n = f.n[2];
    za.n_t = f.n_t;
    za.row_stride = ws;
    za.lo = f.lo[2];
    za.hi = f.hi[2];
    e = dispatch_zpass<T>(f.p_s, za, s);
    if (e != cudaSuccess) return e;
  }
  // time
  TArgs<T> ta{};
  ta.Ms = Ms;
  ta.Js = Js;
  ta.ls_last = f.ls_last;
  ta.y = y;
  ta.bK = f.bKt;
  ta.bM = f.bMt;
  ta.outer = f.B;
  ta.inner = Ns;
  ta.n = f.n_t;
  ta.row_stride = wt;
  ta.lo = f.lo_t;
  ta.hi = f.hi_t;
  ta.fuse = f.fuse;
  return dispatch_tpass<T>(f.p_t, ta, s);
}

template <typename T>
void toeplitz_rows(const T *const *bands, int nbands, int n, int stride, int *lo, int *hi) {
  const int mid = n / 2;
  auto same = [&](int i) {
    for (int b = 0; b < nbands; ++b)
      if (std::memcmp(bands[b] + static_cast<size_t>(i) * stride, bands[b] + static_cast<size_t>(mid) * stride,
                      sizeof(T) * stride) != 0)
        return false;
    return true;
  };
  int l = mid, h = mid + 1;
  while (l > 0 && same(l - 1)) --l;
  while (h < n && same(h)) ++h;
  *lo = n > 0 ? l : 0;
  *hi = n > 0 ? h : 0;
}
template void toeplitz_rows<double>(const double *const *, int, int, int, int *, int *);
template void toeplitz_rows<float>(const float *const *, int, int, int, int *, int *);
template void toeplitz_rows<dfloat>(const dfloat *const *, int, int, int, int *, int *);

template cudaError_t launch_fused_A<double>(const FusedA<double> &, const double *, double *, cudaStream_t);
template cudaError_t launch_fused_A<float>(const FusedA<float> &, const float *, float *, cudaStream_t);
template cudaError_t launch_fused_A<dfloat>(const FusedA<dfloat> &, const dfloat *, dfloat *, cudaStream_t);

cudaError_t launch_df_split(const double *x, dfloat *y, long long N, int B, const CGState *scale, cudaStream_t s) {
  if (N < 0 || B < 1 || B > 65535) return cudaErrorInvalidValue;
  if (N > 0) df_split_kernel<<<dim3(df_grid(N), B), kDfThreads, 0, s>>>(x, y, N, scale);
  return cudaGetLastError();
}
cudaError_t launch_df_join(const dfloat *y, double *x, long long N, int B, const CGState *scale, cudaStream_t s) {
  if (N < 0 || B < 1 || B > 65535) return cudaErrorInvalidValue;
  if (N > 0) df_join_kernel<<<dim3(df_grid(N), B), kDfThreads, 0, s>>>(y, x, N, scale);
  return cudaGetLastError();
}

}  // namespace stls
