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
#include "kernels.h"

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

// ---- directions 1 and 2 --------------------------------------------------------------
// Columns are the (slice, i_1) pairs in order; a CTA owns kAThreads consecutive
// columns and walks i_2.  Each row i_2 of the CTA's columns (plus P columns of
// halo on each side) is staged in shared memory; every thread forms the
// direction-1 products M1 x, J1 x, K1 x of its column from its 2P+1 neighbours
// (neighbours in another slice are masked), keeps them in a window of 2P+1
// rows, and emits the direction-2 outputs of the row P behind.
template <typename T, int P>
__global__ void __launch_bounds__(kAThreads) slice_kernel(const __grid_constant__ SliceArgs<T> a) {
  constexpr int W = 2 * P + 1, D = prefetch_rows<T>(), R = D + 1, RW = kAThreads + 2 * P;
  __shared__ __align__(16) T ring[R][RW];
  const int tid = threadIdx.x, n1 = a.n1, n2 = a.n2, wp = a.row_stride;
  const long long area = static_cast<long long>(n1) * n2;
  const long long ncols = a.slices * n1;
  const long long c0 = static_cast<long long>(blockIdx.x) * kAThreads;
  const long long col = c0 + tid;
  const bool active = col < ncols;
  const long long s = active ? col / n1 : 0;
  const int x = active ? static_cast<int>(col - s * n1) : 0;
  const long long own = active ? s * area + x : 0;
  long long halo = 0;
  bool has_halo = false;
  int hslot = 0;
  if (tid < 2 * P) {
    const long long hc = tid < P ? c0 - P + tid : c0 + kAThreads + (tid - P);
    hslot = tid < P ? tid : kAThreads + tid;
    if (hc >= 0 && hc < ncols) {
      const long long hs = hc / n1;
      halo = hs * area + (hc - hs * n1);
      has_halo = true;
    }
  }
  unsigned valid = 0;  // bit w: neighbour i_1 = x - P + w lies in this slice
#pragma unroll
  for (int w = 0; w < W; ++w)
    if (x - P + w >= 0 && x - P + w < n1) valid |= 1u << w;
  T cM[W], cJ[W], cK[W];
  load_row<T, W>(a.bM1 + static_cast<size_t>(x) * wp, cM);
  load_row<T, W>(a.bJ1 + static_cast<size_t>(x) * wp, cJ);
  load_row<T, W>(a.bK1 + static_cast<size_t>(x) * wp, cK);
  const T *__restrict__ X = a.x;
  // row y of this CTA's columns (and halo) into ring slot y % R, one commit group per row
  auto issue = [&](int y) {
    if (y < n2) {
      T *row = ring[y % R];
      cp_async_elem(row + P + tid, X + own + static_cast<long long>(y) * n1, active);
      if (tid < 2 * P) cp_async_elem(row + hslot, X + halo + static_cast<long long>(y) * n1, has_halo);
    }
    cp_async_commit();
  };
#pragma unroll
  for (int e = 0; e < D; ++e) issue(e);
  T wm[W], wj[W], wk[W];
#pragma unroll
  for (int w = 0; w < W; ++w) wm[w] = wj[w] = wk[w] = T(0);
  const bool ls_row = a.ls_last != nullptr && active && (s % a.n_t) == a.n_t - 1;
  for (int yy = 0; yy < n2 + P; ++yy) {
    // Row yy has landed once at most D - 1 younger groups are pending; the
    // barrier publishes every thread's copies.  Slot (yy + D) % R, refilled
    // below, was last read at row yy - 1, before this barrier.
    cp_async_wait<D - 1>();
    __syncthreads();
    T m0 = T(0), j0 = T(0), k0 = T(0);
    if (yy < n2) {
      const T *row = ring[yy % R];
      T v[W];
#pragma unroll
      for (int w = 0; w < W; ++w) v[w] = ((valid >> w) & 1u) ? row[tid + w] : T(0);
      m0 = band_dot(cM, v, T(0));
      j0 = band_dot(cJ, v, T(0));
      k0 = band_dot(cK, v, T(0));
    }
    issue(yy + D);
    slide(wm, m0);
    slide(wj, j0);
    slide(wk, k0);
    const int y = yy - P;
    if (y >= 0 && active) {
      const size_t r = static_cast<size_t>(y) * wp;
      T c[W];
      load_row<T, W>(a.bM2 + r, c);
      const T om = band_dot(c, wm, T(0));
      T oj = band_dot(c, wj, T(0));
      T ok = T(0);
      if (a.ls_last == nullptr || ls_row) ok = band_dot(c, wk, T(0));
      load_row<T, W>(a.bJ2 + r, c);
      oj = band_dot(c, wm, oj);
      load_row<T, W>(a.b2K2 + r, c);
      oj = band_dot(c, wk, oj);
      const long long off = own + static_cast<long long>(y) * n1;
      a.out_m[off] = om;
      a.out_j[off] = oj;
      if (a.ls_last == nullptr || ls_row) {
        load_row<T, W>(a.bK2 + r, c);
        ok = band_dot(c, wm, ok);
        if (a.ls_last == nullptr)
          a.out_k[off] = ok;
        else
          a.ls_last[(s / a.n_t) * area + static_cast<long long>(y) * n1 + x] = ok;
      }
    }
  }
  cp_async_wait<0>();
}

// ---- direction 3 ------------------------------------------------------------------------
// One thread per (b, t, i_1, i_2) column, walking i_3 with a register window
// for each of m, j', k and a ring of D rows already in flight.
template <typename T, int P>
__global__ void __launch_bounds__(kAThreads) zpass_kernel(const __grid_constant__ ZArgs<T> a) {
  constexpr int W = 2 * P + 1, D = prefetch_rows<T>();
  // thread-private rings: ring[slot][input][thread]
  __shared__ __align__(16) T ring[D][3][kAThreads];
  const int tid = threadIdx.x;
  const long long col = static_cast<long long>(blockIdx.x) * kAThreads + tid;
  if (col >= a.outer * a.inner) return;  // no block-wide barrier below
  const long long inner = a.inner, o = col / inner, cc = col - o * inner;
  const int n = a.n, wp = a.row_stride;
  const long long base = o * n * inner + cc;
  const T *__restrict__ Im = a.m + base;
  const T *__restrict__ Ij = a.j + base;
  const T *__restrict__ Ik = a.k + base;
  auto ld = [&](const T *__restrict__ p, int r) -> T { return (r >= 0 && r < n) ? p[r * inner] : T(0); };
  // row r (>= P + 1) into slot r % D, one commit group per row
  auto issue = [&](int r) {
    const bool ok = r < n;
    const long long off = ok ? static_cast<long long>(r) * inner : 0;
    cp_async_elem(&ring[r % D][0][tid], Im + off, ok);
    cp_async_elem(&ring[r % D][1][tid], Ij + off, ok);
    cp_async_elem(&ring[r % D][2][tid], Ik + off, ok);
    cp_async_commit();
  };
#pragma unroll
  for (int e = 0; e < D; ++e) issue(P + 1 + e);
  T wm[W], wj[W], wk[W];
#pragma unroll
  for (int w = 0; w < W; ++w) {
    wm[w] = ld(Im, w - P);
    wj[w] = ld(Ij, w - P);
    wk[w] = ld(Ik, w - P);
  }
  const bool ls_col = a.ls_last != nullptr && (o % a.n_t) == a.n_t - 1;
  T *ls = ls_col ? a.ls_last + (o / a.n_t) * n * inner + cc : nullptr;
  for (int i = 0; i < n; ++i) {
    const size_t r = static_cast<size_t>(i) * wp;
    T c[W];
    load_row<T, W>(a.bM + r, c);
    const T oms = band_dot(c, wm, T(0));
    T ojs = band_dot(c, wj, T(0));
    T ols = T(0);
    if (ls_col) ols = band_dot(c, wk, T(0));
    load_row<T, W>(a.bJ + r, c);
    ojs = band_dot(c, wm, ojs);
    load_row<T, W>(a.b2K + r, c);
    ojs = band_dot(c, wk, ojs);
    a.Ms[base + static_cast<long long>(i) * inner] = oms;
    a.Js[base + static_cast<long long>(i) * inner] = ojs;
    if (ls_col) {
      load_row<T, W>(a.bK + r, c);
      ls[static_cast<long long>(i) * inner] = band_dot(c, wm, ols);
    }
    // the window takes row i + P + 1 (its group is the oldest of the D pending)
    cp_async_wait<D - 1>();
    const int nr = i + P + 1, sl = nr % D;
    slide(wm, ring[sl][0][tid]);
    slide(wj, ring[sl][1][tid]);
    slide(wk, ring[sl][2][tid]);
    issue(nr + D);
  }
  cp_async_wait<0>();
}

// ---- time direction -------------------------------------------------------------------
// y = K_t (x) (M_s x) + M_t (x) (J_s x), and + L_s x on the last time slice.
template <typename T, int P>
__global__ void __launch_bounds__(kAThreads) tpass_kernel(const __grid_constant__ TArgs<T> a) {
  constexpr int W = 2 * P + 1, D = prefetch_rows<T>();
  __shared__ __align__(16) T ring[D][2][kAThreads];
  const int tid = threadIdx.x;
  const long long col = static_cast<long long>(blockIdx.x) * kAThreads + tid;
  if (col >= a.outer * a.inner) return;  // no block-wide barrier below
  const long long inner = a.inner, o = col / inner, cc = col - o * inner;
  const int n = a.n, wp = a.row_stride;
  const long long base = o * n * inner + cc;
  const T *__restrict__ Ims = a.Ms + base;
  const T *__restrict__ Ijs = a.Js + base;
  auto ld = [&](const T *__restrict__ p, int r) -> T { return (r >= 0 && r < n) ? p[r * inner] : T(0); };
  auto issue = [&](int r) {
    const bool ok = r < n;
    const long long off = ok ? static_cast<long long>(r) * inner : 0;
    cp_async_elem(&ring[r % D][0][tid], Ims + off, ok);
    cp_async_elem(&ring[r % D][1][tid], Ijs + off, ok);
    cp_async_commit();
  };
#pragma unroll
  for (int e = 0; e < D; ++e) issue(P + 1 + e);
  T wm[W], wj[W];
#pragma unroll
  for (int w = 0; w < W; ++w) {
    wm[w] = ld(Ims, w - P);
    wj[w] = ld(Ijs, w - P);
  }
  for (int i = 0; i < n; ++i) {
    const size_t r = static_cast<size_t>(i) * wp;
    T c[W];
    load_row<T, W>(a.bK + r, c);
    T out = band_dot(c, wm, T(0));
    load_row<T, W>(a.bM + r, c);
    out = band_dot(c, wj, out);
    if (i == n - 1) out += a.ls_last[o * inner + cc];
    a.y[base + static_cast<long long>(i) * inner] = out;
    cp_async_wait<D - 1>();
    const int nr = i + P + 1, sl = nr % D;
    slide(wm, ring[sl][0][tid]);
    slide(wj, ring[sl][1][tid]);
    issue(nr + D);
  }
  cp_async_wait<0>();
}

long long blocks_for(long long cols) { return (cols + kAThreads - 1) / kAThreads; }

template <typename T, int P>
cudaError_t launch_slice_p(const SliceArgs<T> &a, cudaStream_t s) {
  const long long g = blocks_for(a.slices * a.n1);
  if (g > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  if (g > 0) slice_kernel<T, P><<<static_cast<unsigned>(g), kAThreads, 0, s>>>(a);
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
  const long long g = blocks_for(a.outer * a.inner);
  if (g > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  if (g > 0) tpass_kernel<T, P><<<static_cast<unsigned>(g), kAThreads, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t dispatch_slice(int p, const SliceArgs<T> &a, cudaStream_t s) {
  switch (p) {
    case 1: return launch_slice_p<T, 1>(a, s);
    case 2: return launch_slice_p<T, 2>(a, s);
    case 3: return launch_slice_p<T, 3>(a, s);
    case 4: return launch_slice_p<T, 4>(a, s);
    case 5: return launch_slice_p<T, 5>(a, s);
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
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

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
  sa.n1 = f.n[0];
  sa.n2 = f.n[1];
  sa.n_t = f.n_t;
  sa.row_stride = ws;
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
  return dispatch_tpass<T>(f.p_t, ta, s);
}

template cudaError_t launch_fused_A<double>(const FusedA<double> &, const double *, double *, cudaStream_t);
template cudaError_t launch_fused_A<float>(const FusedA<float> &, const float *, float *, cudaStream_t);

}  // namespace stls
