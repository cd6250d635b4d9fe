// FP64 vector kernels of the (flexible) preconditioned CG method and their
// inner products (Sec. 4.2: CG on the SPD system; Sec. 5: tolerance on the
// relative residual, zero initial guess).
//
// Reductions are deterministic: every block of the (grid x batch) launch
// writes its partial sums, and the last block to finish (atomic ticket) adds
// the partials in index order and updates the per-right-hand-side CG scalars
// on the device.  No kernel waits on another block.
#include <cmath>

#include "dot2f.cuh"
#include "kernels.h"
#include "tc_ptx.cuh"

namespace stls {

namespace {

constexpr int kThreads = 256;
// Grid-stride loops handle kU entries per trip, S apart: every load of the
// trip is issued before any of them is used, so that a thread keeps kU loads
// of each vector in flight (a streaming kernel needs about 45 GB/s per SM,
// i.e. tens of KB in flight).  The entries are still visited, and summed, in
// the order i0, i0 + S, i0 + 2S, ..., so results do not depend on kU.
constexpr int kU = 4;
// Resident blocks per SM the kernels are compiled for (64 registers a thread:
// room for the kU loads of up to four vectors).
constexpr int kBlocksPerSM = 4;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sums of NV values, result valid in thread 0.
template <int NV>
__device__ void block_sum(double (&v)[NV]) {
  __shared__ double sh[NV][kThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double s = warp_sum(v[k]);
    if (lane == 0) sh[k][wid] = s;
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = lane < kThreads / 32 ? sh[k][lane] : 0.0;
      v[k] = warp_sum(s);
    }
  }
  __syncthreads();
}

// Writes this block's partial sums; returns true in every thread of the last
// block of this right-hand side, with `tot` holding the ordered total.
template <int NV>
__device__ bool grid_sum(double (&v)[NV], RedWork rw, int b, double (&tot)[NV]) {
  __shared__ bool is_last;
  block_sum<NV>(v);
  if (threadIdx.x == 0) {
    double *dst = rw.partials + (static_cast<size_t>(b) * rw.grid + blockIdx.x) * 2;
#pragma unroll
    for (int k = 0; k < NV; ++k) dst[k] = v[k];
    __threadfence();
    unsigned t = atomicAdd(rw.tickets + b, 1u);
    is_last = (t == static_cast<unsigned>(rw.grid - 1));
  }
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  double s[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) s[k] = 0.0;
  const volatile double *src = rw.partials + static_cast<size_t>(b) * rw.grid * 2;
  for (int g = threadIdx.x; g < rw.grid; g += kThreads)
#pragma unroll
    for (int k = 0; k < NV; ++k) s[k] += src[g * 2 + k];
  block_sum<NV>(s);
  if (threadIdx.x == 0) rw.tickets[b] = 0u;
#pragma unroll
  for (int k = 0; k < NV; ++k) tot[k] = s[k];
  return true;
}

__global__ void __launch_bounds__(kThreads, kBlocksPerSM)
    cg_init_kernel(const double *__restrict__ F, double *__restrict__ x, double *__restrict__ r,
                   long long N, CGState *st, RedWork rw) {
  const int b = blockIdx.y;
  const double *Fb = F + static_cast<size_t>(b) * N;
  double *xb = x + static_cast<size_t>(b) * N, *rb = r + static_cast<size_t>(b) * N;
  double v[1] = {0.0};
  const long long i0 = blockIdx.x * static_cast<long long>(kThreads) + threadIdx.x;
  const long long S = static_cast<long long>(gridDim.x) * kThreads;
  for (long long i = i0; i < N; i += kU * S) {
    double f[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u)
      if (i + u * S < N) f[u] = Fb[i + u * S];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const long long j = i + u * S;
      if (j < N) {
        xb[j] = 0.0;
        rb[j] = f[u];
        v[0] = fma(f[u], f[u], v[0]);
      }
    }
  }
  double tot[1];
  if (grid_sum<1>(v, rw, b, tot) && threadIdx.x == 0) {
    CGState &s = st[b];
    s.nF2 = tot[0];
    s.rr = tot[0];
    s.iters = 0;
    s.df_iters = 0;
    s.status = 0;
    s.rel_res = 1.0;
    s.true_rr = 0.0;
    s.alpha = s.beta = s.pq = s.rz = 0.0;
    s.active = 1;
    if (!isfinite(tot[0])) {
      s.status = STLS_ENONFINITE;
      s.active = 0;
    } else if (tot[0] == 0.0) {
      s.rel_res = 0.0;
      s.active = 0;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads, kBlocksPerSM)
    cg_alpha_kernel(const T *__restrict__ p, const T *__restrict__ q, long long N,
                    CGState *st, RedWork rw) {
  const int b = blockIdx.y;
  const T *pb = p + static_cast<size_t>(b) * N, *qb = q + static_cast<size_t>(b) * N;
  double v[1] = {0.0};
  if constexpr (sizeof(T) == 4) {
    Dot2f acc;
    for (long long i = blockIdx.x * static_cast<long long>(kThreads) + threadIdx.x; i < N;
         i += static_cast<long long>(gridDim.x) * kThreads)
      acc.add(pb[i], qb[i]);
    v[0] = acc.value();
  } else {
    for (long long i = blockIdx.x * static_cast<long long>(kThreads) + threadIdx.x; i < N;
         i += static_cast<long long>(gridDim.x) * kThreads)
      v[0] = fma(static_cast<double>(pb[i]), static_cast<double>(qb[i]), v[0]);
  }
  double tot[1];
  if (grid_sum<1>(v, rw, b, tot) && threadIdx.x == 0) {
    CGState &s = st[b];
    if (!s.active) return;
    s.pq = tot[0];
    if (!isfinite(tot[0])) {
      s.status = STLS_ENONFINITE;
      s.active = 0;
    } else if (!(tot[0] > 0.0)) {
      s.status = STLS_EBREAKDOWN;
      s.active = 0;
    } else {
      s.alpha = s.rz / tot[0];
    }
  }
}

// PadOut (FP32 only): also writes r rounded to TF32 into rows of `pad.n`
// values `pad.np` apart (the TF32 preconditioner's first input), so that the
// preconditioner needs no padding pass.
struct PadOut {
  float *out;
  int n, np;
};

// Offset of entry i of one right-hand side in the padded rows
// (i + (i / n)(np - n)), for i = i0, i0 + S, i0 + 2S, ..., without divisions.
struct PadIter {
  unsigned off = 0, soff = 0;
  int col = 0, scol = 0, n = 1, gap = 0;
  __device__ __forceinline__ PadIter(long long i0, long long S, const PadOut &p) {
    const long long row = i0 / p.n, srow = S / p.n;
    n = p.n;
    gap = p.np - p.n;
    col = static_cast<int>(i0 - row * p.n);
    scol = static_cast<int>(S - srow * p.n);
    off = static_cast<unsigned>(row * p.np + col);
    soff = static_cast<unsigned>(srow * p.np + scol);
  }
  __device__ __forceinline__ void next() {
    off += soff;
    col += scol;
    if (col >= n) {
      col -= n;
      off += gap;
    }
  }
};

// (kBlocksPerSM blocks of 256 threads per SM: the reduction grid is sized for that)
// DEFER: x += alpha p is left to the next p update (launch_cg_p with x), or to
// launch_ir_correct once the loop ends; xpend records that it is owed.
template <typename T, bool PAD = false, bool DEFER = false>
__global__ void __launch_bounds__(kThreads, kBlocksPerSM)
    cg_xr_kernel(T *__restrict__ x, T *__restrict__ r, const T *__restrict__ p,
                 const T *__restrict__ q, long long N, double tol, CGState *st, RedWork rw, PadOut pad = {}) {
  const int b = blockIdx.y;
  const bool active = st[b].active != 0;
  const T alpha = static_cast<T>(st[b].alpha);
  T *xb = x + static_cast<size_t>(b) * N, *rb = r + static_cast<size_t>(b) * N;
  const T *pb = p + static_cast<size_t>(b) * N, *qb = q + static_cast<size_t>(b) * N;
  double v[1] = {0.0};
  if (active) {
    const long long i0 = blockIdx.x * static_cast<long long>(kThreads) + threadIdx.x;
    const long long S = static_cast<long long>(gridDim.x) * kThreads;
    if constexpr (sizeof(T) == 4) {
      Dot2f acc;
      PadIter it(i0, S, PAD ? pad : PadOut{nullptr, 1, 1});
      float *pb_out = PAD ? pad.out + static_cast<size_t>(b) * (N / pad.n) * pad.np : nullptr;
      for (long long i = i0; i < N; i += kU * S) {
        T xv[kU], pv[kU], qv[kU], rv[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          const long long j = i + u * S;
          if (j < N) {
            if (!DEFER) {
              xv[u] = xb[j];
              pv[u] = pb[j];
            }
            qv[u] = qb[j];
            rv[u] = rb[j];
          }
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          const long long j = i + u * S;
          if (j < N) {
            if (!DEFER) xb[j] = fma(alpha, pv[u], xv[u]);
            const T ri = fma(-alpha, qv[u], rv[u]);
            rb[j] = ri;
            acc.add(ri, ri);
            if (PAD) {
              pb_out[it.off] = ptx::tf32_rna(ri);
              it.next();
            }
          }
        }
      }
      v[0] = acc.value();
    } else {
      for (long long i = i0; i < N; i += kU * S) {
        T xv[kU], pv[kU], qv[kU], rv[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          const long long j = i + u * S;
          if (j < N) {
            xv[u] = xb[j];
            pv[u] = pb[j];
            qv[u] = qb[j];
            rv[u] = rb[j];
          }
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          const long long j = i + u * S;
          if (j < N) {
            xb[j] = fma(alpha, pv[u], xv[u]);
            const T ri = fma(-alpha, qv[u], rv[u]);
            rb[j] = ri;
            v[0] = fma(static_cast<double>(ri), static_cast<double>(ri), v[0]);
          }
        }
      }
    }
  }
  double tot[1];
  if (grid_sum<1>(v, rw, b, tot) && threadIdx.x == 0) {
    CGState &s = st[b];
    if (!s.active) return;
    s.iters += 1;
    if (DEFER) s.xpend = 1;
    s.rr = tot[0];
    s.rel_res = sqrt(tot[0] / s.nF2);
    if (!isfinite(tot[0])) {
      s.status = STLS_ENONFINITE;
      s.active = 0;
    } else if (s.rel_res <= (tol >= 0.0 ? tol : s.tol_in)) {
      s.active = 0;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads, kBlocksPerSM)
    cg_beta_kernel(const T *__restrict__ z, const T *__restrict__ r,
                   const T *__restrict__ q, long long N, int flexible, int first, CGState *st,
                   RedWork rw) {
  const int b = blockIdx.y;
  if (first < 0) first = st[b].iters == 0;
  const T *zb = z + static_cast<size_t>(b) * N, *rb = r + static_cast<size_t>(b) * N;
  const T *qb = q + static_cast<size_t>(b) * N;
  const bool need_zq = flexible && !first;
  double v[2] = {0.0, 0.0};
  const long long i0 = blockIdx.x * static_cast<long long>(kThreads) + threadIdx.x;
  const long long S = static_cast<long long>(gridDim.x) * kThreads;
  if constexpr (sizeof(T) == 4) {
    Dot2f zr, zq;
    for (long long i = i0; i < N; i += kU * S) {
      T zv[kU], rv[kU], qv[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const long long j = i + u * S;
        if (j < N) {
          zv[u] = zb[j];
          rv[u] = rb[j];
          if (need_zq) qv[u] = qb[j];
        }
      }
#pragma unroll
      for (int u = 0; u < kU; ++u)
        if (i + u * S < N) {
          zr.add(zv[u], rv[u]);
          if (need_zq) zq.add(zv[u], qv[u]);
        }
    }
    v[0] = zr.value();
    v[1] = zq.value();
  } else {
    for (long long i = i0; i < N; i += kU * S) {
      T zv[kU], rv[kU], qv[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const long long j = i + u * S;
        if (j < N) {
          zv[u] = zb[j];
          rv[u] = rb[j];
          if (need_zq) qv[u] = qb[j];
        }
      }
#pragma unroll
      for (int u = 0; u < kU; ++u)
        if (i + u * S < N) {
          const double zi = static_cast<double>(zv[u]);
          v[0] = fma(zi, static_cast<double>(rv[u]), v[0]);
          if (need_zq) v[1] = fma(zi, static_cast<double>(qv[u]), v[1]);
        }
    }
  }
  double tot[2];
  if (grid_sum<2>(v, rw, b, tot) && threadIdx.x == 0) {
    CGState &s = st[b];
    if (!s.active) return;
    const double zr = tot[0];
    if (!isfinite(zr) || !isfinite(tot[1])) {
      s.status = STLS_ENONFINITE;
      s.active = 0;
      return;
    }
    if (!(zr > 0.0)) {
      s.status = STLS_EBREAKDOWN;
      s.active = 0;
      return;
    }
    if (first) {
      s.beta = 0.0;
    } else if (flexible) {
      // beta = (z_{k+1}, r_{k+1} - r_k) / (z_k, r_k) with r_{k+1} - r_k = -alpha q
      s.beta = -s.alpha * tot[1] / s.rz;
    } else {
      s.beta = zr / s.rz;
    }
    s.rz = zr;
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads, kBlocksPerSM)
    cg_p_kernel(const T *__restrict__ z, T *__restrict__ p, long long N, int first,
                CGState *st, T *__restrict__ x, unsigned *tickets) {
  const int b = blockIdx.y;
  if (!st[b].active) return;
  if (first < 0) first = st[b].iters == 0;
  const T beta = static_cast<T>(st[b].beta);
  const T *zb = z + static_cast<size_t>(b) * N;
  T *pb = p + static_cast<size_t>(b) * N;
  if (x != nullptr && !first) {
    // the x update deferred by cg_xr: x += alpha p with the p it used
    const T alpha = static_cast<T>(st[b].alpha);
    T *xb = x + static_cast<size_t>(b) * N;
    const long long i0 = blockIdx.x * static_cast<long long>(kThreads) + threadIdx.x;
    const long long S = static_cast<long long>(gridDim.x) * kThreads;
    for (long long i = i0; i < N; i += kU * S) {
      T pv[kU], xv[kU], zv[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const long long j = i + u * S;
        if (j < N) {
          pv[u] = pb[j];
          xv[u] = xb[j];
          zv[u] = zb[j];
        }
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const long long j = i + u * S;
        if (j < N) {
          xb[j] = fma(alpha, pv[u], xv[u]);
          pb[j] = fma(beta, pv[u], zv[u]);
        }
      }
    }
    // the last block clears the flag (every block has read the state by then)
    __shared__ bool is_last;
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      is_last = atomicAdd(tickets + b, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (is_last && threadIdx.x == 0) {
      st[b].xpend = 0;
      tickets[b] = 0u;
    }
    return;
  }
  const long long i0 = blockIdx.x * static_cast<long long>(kThreads) + threadIdx.x;
  const long long S = static_cast<long long>(gridDim.x) * kThreads;
  for (long long i = i0; i < N; i += kU * S) {
    T pv[kU], zv[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const long long j = i + u * S;
      if (j < N) {
        zv[u] = zb[j];
        if (!first) pv[u] = pb[j];
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const long long j = i + u * S;
      if (j < N) pb[j] = first ? zv[u] : fma(beta, pv[u], zv[u]);
    }
  }
}

__global__ void __launch_bounds__(kThreads, kBlocksPerSM)
    true_residual_kernel(const double *__restrict__ F, const double *__restrict__ Ax, long long N,
                         CGState *st, RedWork rw) {
  const int b = blockIdx.y;
  const double *Fb = F + static_cast<size_t>(b) * N, *Ab = Ax + static_cast<size_t>(b) * N;
  double v[1] = {0.0};
  for (long long i = blockIdx.x * static_cast<long long>(kThreads) + threadIdx.x; i < N;
       i += static_cast<long long>(gridDim.x) * kThreads) {
    double e = Fb[i] - Ab[i];
    v[0] = fma(e, e, v[0]);
  }
  double tot[1];
  if (grid_sum<1>(v, rw, b, tot) && threadIdx.x == 0) st[b].true_rr = tot[0];
}

// Refinement form: inner right-hand side r32 = r64 2^-k (FP32, rounded to
// nearest; ||r64|| = f 2^k with f in [0.5, 1), so the power-of-two scaling is
// exact and done on the exponent field), d = 0, and the inner CG state for it
// (active where the outer solve is active).  No FP64 arithmetic per entry: the
// norm is accumulated by Dot2f.
__global__ void __launch_bounds__(kThreads, kBlocksPerSM)
    ir_start_kernel(const double *__restrict__ r64, float *__restrict__ r32, float *__restrict__ d,
                    long long N, const CGState *outer, CGState *inner, RedWork rw, PadOut pad, double eta,
                    int limit) {
  const int b = blockIdx.y;
  const int k = ptx::df_scale_exp(outer[b].rr);
  const double *rb = r64 + static_cast<size_t>(b) * N;
  float *ib = r32 + static_cast<size_t>(b) * N, *db = d + static_cast<size_t>(b) * N;
  Dot2f acc;
  const long long i0 = blockIdx.x * static_cast<long long>(kThreads) + threadIdx.x;
  const long long S = static_cast<long long>(gridDim.x) * kThreads;
  const bool padded = pad.out != nullptr;
  PadIter it(i0, S, padded ? pad : PadOut{nullptr, 1, 1});
  float *pb_out = padded ? pad.out + static_cast<size_t>(b) * (N / pad.n) * pad.np : nullptr;
  for (long long i = i0; i < N; i += kU * S) {
    double rv[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u)
      if (i + u * S < N) rv[u] = rb[i + u * S];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const long long j = i + u * S;
      if (j < N) {
        const float x = ptx::f64_to_f32_rn(ptx::scale_f64(rv[u], -k));
        ib[j] = x;
        db[j] = 0.f;
        acc.add(x, x);
        if (padded) {
          pb_out[it.off] = ptx::tf32_rna(x);
          it.next();
        }
      }
    }
  }
  double v[1] = {acc.value()};
  double tot[1];
  if (grid_sum<1>(v, rw, b, tot) && threadIdx.x == 0) {
    CGState &s = inner[b];
    s.nF2 = tot[0];
    s.rr = tot[0];
    s.iters = 0;
    s.xpend = 0;
    s.status = 0;
    s.rel_res = 1.0;
    s.alpha = s.beta = s.pq = s.rz = 0.0;
    s.tol_in = eta;
    s.limit = limit;
    s.active = outer[b].active && tot[0] > 0.0;
  }
}

__global__ void inner_cond_kernel(const CGState *st, int B, const int *err, cudaGraphConditionalHandle h) {
  unsigned go = 0;
  for (int b = 0; b < B; ++b)
    if (st[b].active && st[b].iters < st[b].limit) go = 1;
  if (err != nullptr && *reinterpret_cast<const volatile int *>(err) != 0) go = 0;
  cudaGraphSetConditional(h, go);
}

// u += 2^k d (the scaling of ir_start undone exactly) for the right-hand sides
// whose outer solve is active; one FP64 add per entry.  With udf != NULL also
// the double-float image of the new u (launch_df_split's, scaled by the
// exponent of ||F||), for every right-hand side.
__global__ void __launch_bounds__(kThreads, kBlocksPerSM)
    ir_correct_kernel(double *__restrict__ u, const float *__restrict__ d, const float *__restrict__ p,
                      const CGState *inner, dfloat *__restrict__ udf, long long N, const CGState *outer) {
  const int b = blockIdx.y;
  const bool active = outer[b].active != 0;
  if (!active && udf == nullptr) return;
  // the inner solve's last x += alpha p, when its CG update deferred it
  const bool pend = active && p != nullptr && inner[b].xpend != 0;
  const float alpha = pend ? static_cast<float>(inner[b].alpha) : 0.f;
  const float *pb = p != nullptr ? p + static_cast<size_t>(b) * N : nullptr;
  const int k = ptx::df_scale_exp(outer[b].rr), kF = ptx::df_scale_exp(outer[b].nF2);
  double *ub = u + static_cast<size_t>(b) * N;
  const float *db = d + static_cast<size_t>(b) * N;
  dfloat *yb = udf != nullptr ? udf + static_cast<size_t>(b) * N : nullptr;
  const long long i0 = blockIdx.x * static_cast<long long>(kThreads) + threadIdx.x;
  const long long S = static_cast<long long>(gridDim.x) * kThreads;
  for (long long i = i0; i < N; i += kU * S) {
    double uv[kU];
    float dv[kU], pv[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const long long j = i + u * S;
      if (j < N) {
        uv[u] = ub[j];
        if (active) dv[u] = db[j];
        if (pend) pv[u] = pb[j];
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const long long j = i + u * S;
      if (j >= N) continue;
      double v = uv[u];
      if (active) {
        if (pend) dv[u] = fmaf(alpha, pv[u], dv[u]);  // the pending update's own FP32 FMA
        v += ptx::scale_f64(ptx::f32_to_f64(dv[u]), k);
        ub[j] = v;
      }
      if (yb != nullptr) {
        const double w = ptx::scale_f64(v, -kF);
        dfloat o;
        o.h = ptx::f64_to_f32_rn(w);
        o.l = ptx::f64_to_f32_rn(w - ptx::f32_to_f64(o.h));
        yb[j] = o;
      }
    }
  }
}

// r64 = F - A u in FP64 and the outer convergence test on ||r64|| / ||F||
// (`count`: whether this residual ends an outer step).
__global__ void __launch_bounds__(kThreads, kBlocksPerSM)
    ir_residual_kernel(const double *__restrict__ F, const double *__restrict__ Au, double *__restrict__ r64,
                       long long N, double tol, int count, CGState *outer, RedWork rw) {
  const int b = blockIdx.y;
  const double *Fb = F + static_cast<size_t>(b) * N, *Ab = Au + static_cast<size_t>(b) * N;
  double *rb = r64 + static_cast<size_t>(b) * N;
  double v[1] = {0.0};
  const long long i0 = blockIdx.x * static_cast<long long>(kThreads) + threadIdx.x;
  const long long S = static_cast<long long>(gridDim.x) * kThreads;
  for (long long i = i0; i < N; i += kU * S) {
    double fv[kU], av[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const long long j = i + u * S;
      if (j < N) {
        fv[u] = Fb[j];
        av[u] = Ab[j];
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const long long j = i + u * S;
      if (j < N) {
        const double e = fv[u] - av[u];
        rb[j] = e;
        v[0] = fma(e, e, v[0]);
      }
    }
  }
  double tot[1];
  if (grid_sum<1>(v, rw, b, tot) && threadIdx.x == 0) {
    CGState &s = outer[b];
    s.true_rr = tot[0];
    if (!s.active) return;
    s.iters += count;
    s.rr = tot[0];
    s.rel_res = sqrt(tot[0] / s.nF2);
    if (!isfinite(tot[0])) {
      s.status = STLS_ENONFINITE;
      s.active = 0;
    } else if (s.rel_res <= tol) {
      s.active = 0;
    }
  }
}

// r64 = F - 2^k (h + l) for the double-float image h + l of 2^-k A u, in
// FP64 (the FP32 parts are widened and scaled exactly by integer operations),
// and its norm; provisional: no convergence test, no status change.
__global__ void __launch_bounds__(kThreads, kBlocksPerSM)
    ir_residual_df_kernel(const double *__restrict__ F, const dfloat *__restrict__ Au, double *__restrict__ r64,
                          long long N, CGState *outer, RedWork rw) {
  const int b = blockIdx.y;
  const int k = ptx::df_scale_exp(outer[b].nF2);
  const double *Fb = F + static_cast<size_t>(b) * N;
  const dfloat *Ab = Au + static_cast<size_t>(b) * N;
  double *rb = r64 + static_cast<size_t>(b) * N;
  double v[1] = {0.0};
  const long long i0 = blockIdx.x * static_cast<long long>(kThreads) + threadIdx.x;
  const long long S = static_cast<long long>(gridDim.x) * kThreads;
  for (long long i = i0; i < N; i += kU * S) {
    double fv[kU];
    dfloat av[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const long long j = i + u * S;
      if (j < N) {
        fv[u] = Fb[j];
        av[u] = Ab[j];
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const long long j = i + u * S;
      if (j < N) {
        const dfloat a = av[u];
        const double e = (fv[u] - ptx::scale_f64(ptx::f32_to_f64(a.h), k)) - ptx::scale_f64(ptx::f32_to_f64(a.l), k);
        rb[j] = e;
        v[0] = fma(e, e, v[0]);
      }
    }
  }
  double tot[1];
  if (grid_sum<1>(v, rw, b, tot) && threadIdx.x == 0) {
    CGState &s = outer[b];
    s.true_rr = tot[0];
    if (!s.active) return;
    s.iters += 1;
    s.df_iters += 1;
    s.rr = tot[0];
    s.rel_res = sqrt(tot[0] / s.nF2);
  }
}

// out[b] = (x_b, y_b), deterministic like the CG reductions
__global__ void __launch_bounds__(kThreads, kBlocksPerSM)
    vec_dot_kernel(const double *__restrict__ x, const double *__restrict__ y, long long n, double *out, RedWork rw) {
  const int b = blockIdx.y;
  const double *xb = x + static_cast<size_t>(b) * n, *yb = y + static_cast<size_t>(b) * n;
  double v[1] = {0.0};
  const long long i0 = blockIdx.x * static_cast<long long>(kThreads) + threadIdx.x;
  const long long S = static_cast<long long>(gridDim.x) * kThreads;
  for (long long i = i0; i < n; i += kU * S) {
    double xv[kU], yv[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u)
      if (i + u * S < n) {
        xv[u] = xb[i + u * S];
        yv[u] = yb[i + u * S];
      }
#pragma unroll
    for (int u = 0; u < kU; ++u)
      if (i + u * S < n) v[0] = fma(xv[u], yv[u], v[0]);
  }
  double tot[1];
  if (grid_sum<1>(v, rw, b, tot) && threadIdx.x == 0) out[b] = tot[0];
}

__global__ void __launch_bounds__(kThreads, kBlocksPerSM)
    vec_axpby_kernel(const double *__restrict__ ab, const double *x, double *y, long long n) {
  const int b = blockIdx.y, B = gridDim.y;
  const double a = ab[b], c = ab[B + b];
  const double *xb = x + static_cast<size_t>(b) * n;
  double *yb = y + static_cast<size_t>(b) * n;
  for (long long i = blockIdx.x * static_cast<long long>(kThreads) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * kThreads)
    yb[i] = fma(a, xb[i], c * yb[i]);
}

// y[b, i] = x[b, i] w[i] (the diagonal scaling of the geometry-aware preconditioner)
__global__ void __launch_bounds__(kThreads, kBlocksPerSM)
    scale_kernel(const double *x, const double *__restrict__ w, double *y, long long N) {
  const int b = blockIdx.y;
  const double *xb = x + static_cast<size_t>(b) * N;
  double *yb = y + static_cast<size_t>(b) * N;
  for (long long i = blockIdx.x * static_cast<long long>(kThreads) + threadIdx.x; i < N;
       i += static_cast<long long>(gridDim.x) * kThreads)
    yb[i] = xb[i] * w[i];
}

__global__ void lift_combine_kernel(const double *__restrict__ Ls, const double *__restrict__ Js,
                                    const double *__restrict__ e, const double *__restrict__ m,
                                    double *__restrict__ y, long long Ns, int nt) {
  const int b = blockIdx.y;
  const long long N = Ns * nt;
  for (long long i = blockIdx.x * static_cast<long long>(kThreads) + threadIdx.x; i < N;
       i += static_cast<long long>(gridDim.x) * kThreads) {
    long long t = i / Ns, c = i - t * Ns;
    y[b * N + i] = e[t] * Ls[b * Ns + c] + m[t] * Js[b * Ns + c];
  }
}

__global__ void lift_reduce_kernel(const double *__restrict__ lam, const double *__restrict__ g,
                                   const double *__restrict__ e, const double *__restrict__ m,
                                   double *__restrict__ a, double *__restrict__ bs,
                                   double *__restrict__ gs, long long Ns, int nt) {
  const int b = blockIdx.y;
  const long long N = Ns * nt;
  for (long long c = blockIdx.x * static_cast<long long>(kThreads) + threadIdx.x; c < Ns;
       c += static_cast<long long>(gridDim.x) * kThreads) {
    double sa = 0.0, sb = 0.0, sg = 0.0;
    for (int t = 0; t < nt; ++t) {
      double l = lam[b * N + t * Ns + c];
      sa = fma(e[t], l, sa);
      sb = fma(m[t], l, sb);
      sg += g[b * N + t * Ns + c];
    }
    a[b * Ns + c] = sa;
    bs[b * Ns + c] = sb;
    gs[b * Ns + c] = sg;
  }
}

__global__ void axpy_kernel(const double *__restrict__ x, const double *__restrict__ y, double alpha,
                            double *__restrict__ out, long long n) {
  for (long long i = blockIdx.x * static_cast<long long>(kThreads) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * kThreads)
    out[i] = fma(alpha, y[i], x[i]);
}

unsigned grid_1d(long long n) {
  long long g = (n + kThreads - 1) / kThreads;
  if (g > 152 * 16) g = 152 * 16;
  return static_cast<unsigned>(g < 1 ? 1 : g);
}

}  // namespace

int red_grid_for(long long n) {
  // one wave of the reduction kernels: kBlocksPerSM blocks on every SM of the current device
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    sms = 152;
  const long long cap = static_cast<long long>(kBlocksPerSM) * sms;
  long long g = (n + kThreads * kU - 1) / (kThreads * kU);
  if (g > cap) g = cap;
  return static_cast<int>(g < 1 ? 1 : g);
}

cudaError_t launch_cg_init(const double *F, double *x, double *r, long long N, int B, CGState *st,
                           RedWork rw, cudaStream_t s) {
  cg_init_kernel<<<dim3(rw.grid, B), kThreads, 0, s>>>(F, x, r, N, st, rw);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_cg_alpha(const T *p, const T *q, long long N, int B, CGState *st, RedWork rw, cudaStream_t s) {
  cg_alpha_kernel<T><<<dim3(rw.grid, B), kThreads, 0, s>>>(p, q, N, st, rw);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_cg_xr(T *x, T *r, const T *p, const T *q, long long N, int B, double tol, CGState *st,
                         RedWork rw, cudaStream_t s) {
  cg_xr_kernel<T><<<dim3(rw.grid, B), kThreads, 0, s>>>(x, r, p, q, N, tol, st, rw);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_cg_beta(const T *z, const T *r, const T *q, long long N, int B, int flexible, int first,
                           CGState *st, RedWork rw, cudaStream_t s) {
  cg_beta_kernel<T><<<dim3(rw.grid, B), kThreads, 0, s>>>(z, r, q, N, flexible, first, st, rw);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_cg_p(const T *z, T *p, long long N, int B, int first, CGState *st, cudaStream_t s, T *x,
                        unsigned *tickets) {
  if (x != nullptr && tickets == nullptr) return cudaErrorInvalidValue;
  cg_p_kernel<T><<<dim3(grid_1d(N), B), kThreads, 0, s>>>(z, p, N, first, st, x, tickets);
  return cudaGetLastError();
}
#define STLS_INST(T)                                                                                       \
  template cudaError_t launch_cg_alpha<T>(const T *, const T *, long long, int, CGState *, RedWork,       \
                                          cudaStream_t);                                                   \
  template cudaError_t launch_cg_xr<T>(T *, T *, const T *, const T *, long long, int, double, CGState *, \
                                       RedWork, cudaStream_t);                                             \
  template cudaError_t launch_cg_beta<T>(const T *, const T *, const T *, long long, int, int, int,        \
                                         CGState *, RedWork, cudaStream_t);                                \
  template cudaError_t launch_cg_p<T>(const T *, T *, long long, int, int, CGState *, cudaStream_t, T *,  \
                                      unsigned *);
STLS_INST(double)
STLS_INST(float)
#undef STLS_INST
cudaError_t launch_cg_xr_pad(float *x, float *r, const float *p, const float *q, long long N, int B, double tol,
                             CGState *st, RedWork rw, float *rpad, int n0, int np0, int defer, cudaStream_t s) {
  if (n0 < 1 || np0 < n0 || N % n0 != 0 || static_cast<double>(N / n0) * np0 >= 4294967296.0)
    return cudaErrorInvalidValue;
  PadOut pad{rpad, n0, np0};
  if (defer)
    cg_xr_kernel<float, true, true><<<dim3(rw.grid, B), kThreads, 0, s>>>(x, r, p, q, N, tol, st, rw, pad);
  else
    cg_xr_kernel<float, true><<<dim3(rw.grid, B), kThreads, 0, s>>>(x, r, p, q, N, tol, st, rw, pad);
  return cudaGetLastError();
}
cudaError_t launch_ir_start(const double *r64, float *r32, float *d, long long N, int B, const CGState *outer,
                            CGState *inner, RedWork rw, float *rpad, int n0, int np0, double eta, int limit,
                            cudaStream_t s) {
  if (rpad != nullptr && (n0 < 1 || np0 < n0 || N % n0 != 0 || static_cast<double>(N / n0) * np0 >= 4294967296.0))
    return cudaErrorInvalidValue;
  const PadOut pad{rpad, rpad != nullptr ? n0 : 1, rpad != nullptr ? np0 : 1};
  ir_start_kernel<<<dim3(rw.grid, B), kThreads, 0, s>>>(r64, r32, d, N, outer, inner, rw, pad, eta, limit);
  return cudaGetLastError();
}
cudaError_t launch_inner_cond(const CGState *st, int B, const int *err, cudaGraphConditionalHandle h,
                              cudaStream_t s) {
  inner_cond_kernel<<<1, 1, 0, s>>>(st, B, err, h);
  return cudaGetLastError();
}
cudaError_t launch_ir_correct(double *u, const float *d, const float *p, const CGState *inner, dfloat *udf,
                              long long N, int B, const CGState *outer, cudaStream_t s) {
  ir_correct_kernel<<<dim3(grid_1d(N), B), kThreads, 0, s>>>(u, d, p, inner, udf, N, outer);
  return cudaGetLastError();
}
cudaError_t launch_ir_residual(const double *F, const double *Au, double *r64, long long N, int B, double tol,
                               int count, CGState *outer, RedWork rw, cudaStream_t s) {
  ir_residual_kernel<<<dim3(rw.grid, B), kThreads, 0, s>>>(F, Au, r64, N, tol, count, outer, rw);
  return cudaGetLastError();
}
cudaError_t launch_ir_residual_df(const double *F, const dfloat *Au, double *r64, long long N, int B,
                                  CGState *outer, RedWork rw, cudaStream_t s) {
  ir_residual_df_kernel<<<dim3(rw.grid, B), kThreads, 0, s>>>(F, Au, r64, N, outer, rw);
  return cudaGetLastError();
}
cudaError_t launch_true_residual(const double *F, const double *Ax, long long N, int B, CGState *st,
                                 RedWork rw, cudaStream_t s) {
  true_residual_kernel<<<dim3(rw.grid, B), kThreads, 0, s>>>(F, Ax, N, st, rw);
  return cudaGetLastError();
}
cudaError_t launch_lift_combine(const double *Ls, const double *Js, const double *e, const double *m,
                                double *y, long long Ns, int nt, int B, cudaStream_t s) {
  lift_combine_kernel<<<dim3(grid_1d(Ns * nt), B), kThreads, 0, s>>>(Ls, Js, e, m, y, Ns, nt);
  return cudaGetLastError();
}
cudaError_t launch_lift_reduce(const double *lam, const double *g, const double *e, const double *m,
                               double *a, double *bsum, double *gsum, long long Ns, int nt, int B,
                               cudaStream_t s) {
  lift_reduce_kernel<<<dim3(grid_1d(Ns), B), kThreads, 0, s>>>(lam, g, e, m, a, bsum, gsum, Ns, nt);
  return cudaGetLastError();
}
cudaError_t launch_vec_dot(const double *x, const double *y, long long n, int B, double *out, RedWork rw,
                           cudaStream_t s) {
  if (n < 0 || B < 1 || B > 65535) return cudaErrorInvalidValue;
  vec_dot_kernel<<<dim3(rw.grid, B), kThreads, 0, s>>>(x, y, n, out, rw);
  return cudaGetLastError();
}
cudaError_t launch_vec_axpby(const double *ab, const double *x, double *y, long long n, int B, cudaStream_t s) {
  if (n < 0 || B < 1 || B > 65535) return cudaErrorInvalidValue;
  if (n > 0) vec_axpby_kernel<<<dim3(grid_1d(n), B), kThreads, 0, s>>>(ab, x, y, n);
  return cudaGetLastError();
}
cudaError_t launch_scale(const double *x, const double *w, double *y, long long N, int B, cudaStream_t s) {
  if (N < 0 || B < 1 || B > 65535) return cudaErrorInvalidValue;
  if (N > 0) scale_kernel<<<dim3(grid_1d(N), B), kThreads, 0, s>>>(x, w, y, N);
  return cudaGetLastError();
}
cudaError_t launch_axpy(const double *x, const double *y, double alpha, double *out, long long n,
                        cudaStream_t s) {
  axpy_kernel<<<grid_1d(n), kThreads, 0, s>>>(x, y, alpha, out, n);
  return cudaGetLastError();
}

}  // namespace stls
