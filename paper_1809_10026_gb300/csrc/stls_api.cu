// C ABI of the solver (declared in include/stls.h): context creation, the
// matrix-free system matrix (Eq. A_kron), the fast-diagonalization
// preconditioner (Algorithm 1), the PCG / flexible-CG driver and the lifting
// of a non-zero initial datum (Sec. 3.1).
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "kernels.h"
#include "stls_internal.h"
#include "tc_fd.h"

namespace stls {
int copy_factor_public(const HostSetup &hs, int which, int dir, double *out);
}

using stls::BandSpec;
using stls::CGState;
using stls::ModeView;

// Banded factors and state buffers of the matrix-free A x in one precision.
template <typename T>
struct AOps {
  T *band_M[3] = {}, *band_K[3] = {}, *band_J[3] = {};
  T *band_E[3] = {}, *band_Et[3] = {};  // geometry = 1: int (L b_i) b_j g' and its transpose
  T *band_Kt = nullptr, *band_Mt = nullptr;
  // the same bands with rows padded to whole 16-byte vectors, and 2 K (fused A x)
  T *pad_M[3] = {}, *pad_K[3] = {}, *pad_J[3] = {}, *pad_2K[3] = {};
  T *pad_Kt = nullptr, *pad_Mt = nullptr;
  int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0}, lo_t = 0, hi_t = 0;  // identical interior band rows
  T int_Kt[2 * stls::kFusedMaxP + 1] = {}, int_Mt[2 * stls::kFusedMaxP + 1] = {};  // interior time rows (host)
  T int_3[4][2 * stls::kFusedMaxP + 1] = {};  // interior rows of M, J, 2K, K of direction 3 (host)
  T *abuf[8] = {};
  T *ls_buf = nullptr;
};

struct stls_ctx {
  stls::HostSetup hs;
  cudaStream_t stream = nullptr;
  int d = 0, B = 0, n_t = 0;
  int n_s[3] = {1, 1, 1};
  long long Ns = 0, N = 0;
  // device factors
  AOps<double> a64;                 // FP64 A x (residuals, strict forms)
  AOps<float> a32;                  // FP32 A x (inner solves of the refinement form)
  AOps<stls::dfloat> adf;           // double-float A x (provisional outer residuals)
  bool have_df = false;
  double *Uf[4] = {}, *Ub[4] = {};  // U^T (forward) and U (backward), row-major
  double *lam_t = nullptr, *lam_s = nullptr;
  double *e_end = nullptr, *m_int = nullptr;
  double *ones_t = nullptr, *zeros_t = nullptr;  // n_t ones and zeros (u = w + 1 x c0)
  // workspace
  double *r = nullptr, *p = nullptr, *q = nullptr, *z = nullptr;
  double *fd_tmp[2] = {};
  double *lift_tmp[4] = {};
  float *ri = nullptr, *pi = nullptr, *qi = nullptr, *zi = nullptr, *di = nullptr;  // refinement inner vectors
  CGState *st_in = nullptr;
  double *alpha_partials = nullptr;  // fused (p, A p) of the inner solves: B * alpha_blocks(N_s)
  unsigned *alpha_tickets = nullptr;
  double *dF = nullptr, *du = nullptr;
  double *vec_ab = nullptr, *vec_out = nullptr;  // scalars of stls_vec_axpby (2B), results of stls_vec_dot (B)
  double *geo_dinv = nullptr;  // geometry = 1, geo_precond = 0: D^{-1/2} of P^G (N entries)
  double *geo_tmp = nullptr;   // B x N: the scaled input of Pbar^G
  CGState *st = nullptr, *st_host = nullptr;
  stls::RedWork rw{};
  stls::TcFd tc{};
  std::vector<void *> allocations;
  std::vector<std::vector<double>> hist;  // relative residuals of the last solve, per RHS
  long long launches = 0;
  std::string err;
  // inner FP32 loop of the refinement form as a CUDA graph: a while node whose
  // body is one CG step, its condition set on the device (built on first use)
  cudaGraph_t ig_graph = nullptr;
  cudaGraphExec_t ig_exec = nullptr;
  long long ig_body_launches = 0;  // kernels in one body
  bool ig_failed = false;          // the graph could not be built: host-driven loop
  // stls_solve_host: u's copy to the host overlaps the FP64 residual that
  // confirms convergence (side stream); redone if a later step changes u
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_u = nullptr, ev_copied = nullptr;
  bool early_issued = false, early_final = false;
  // timing
  bool timing = false;
  double phase_ms[5] = {0, 0, 0, 0, 0};
  long long phase_count[5] = {0, 0, 0, 0, 0};
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, int>> ev_pairs;  // (phase, first event index)
};

namespace {

thread_local std::string g_create_error;

int set_err(stls_ctx *c, int code, const std::string &msg) {
  if (c != nullptr) c->err = msg;
  return code;
}

int cuda_err(stls_ctx *c, cudaError_t e, const char *where) {
  return set_err(c, STLS_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define STLS_CK(call, where)                              \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_err(c, e_, where); \
  } while (0)

#define STLS_LAUNCH(call, where) \
  do {                           \
    c->launches += 1;            \
    STLS_CK(call, where);        \
  } while (0)

template <typename T>
int dev_alloc(stls_ctx *c, T **ptr, size_t count) {
  void *v = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc(&v, count * sizeof(T));
  if (e != cudaSuccess) return set_err(c, STLS_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  c->allocations.push_back(v);
  *ptr = static_cast<T *>(v);
  return STLS_OK;
}

template <typename T>
int upload(stls_ctx *c, T **ptr, const std::vector<T> &h) {
  int rc = dev_alloc(c, ptr, h.size());
  if (rc) return rc;
  STLS_CK(cudaMemcpy(*ptr, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice), "upload");
  return STLS_OK;
}

// FP64 value in the element type: rounded to nearest for float, split into
// h = fl32(v), l = fl32(v - h) for double-float.
template <typename T>
T to_elem(double v) {
  if constexpr (std::is_same_v<T, stls::dfloat>) {
    stls::dfloat r;
    r.h = static_cast<float>(v);
    r.l = static_cast<float>(v - static_cast<double>(r.h));
    return r;
  } else {
    return static_cast<T>(v);
  }
}

// Band rows (2p+1 values) copied into rows of `stride` values, scaled by `scale`.
template <typename T>
std::vector<T> pad_band(const std::vector<double> &band, int n, int p, int stride, double scale) {
  const int w = 2 * p + 1;
  std::vector<T> out(static_cast<size_t>(n) * stride, T(0));
  for (int i = 0; i < n; ++i)
    for (int o = 0; o < w; ++o) out[static_cast<size_t>(i) * stride + o] = to_elem<T>(scale * band[i * w + o]);
  return out;
}

template <typename T>
int upload_padded(stls_ctx *c, AOps<T> &A, int k, const stls::Dir1D &D, const std::vector<double> &bM,
                  const std::vector<double> &bK, const std::vector<double> &bJ) {
  const int st = stls::band_row_stride(D.p, sizeof(T));
  const std::vector<T> pM = pad_band<T>(bM, D.n, D.p, st, 1.0), pK = pad_band<T>(bK, D.n, D.p, st, 1.0);
  const std::vector<T> pJ = pad_band<T>(bJ, D.n, D.p, st, 1.0), p2K = pad_band<T>(bK, D.n, D.p, st, 2.0);
  const T *all[4] = {pM.data(), pK.data(), pJ.data(), p2K.data()};
  stls::toeplitz_rows<T>(all, 4, D.n, st, &A.lo[k], &A.hi[k]);
  if (k == 2 && A.lo[k] < A.hi[k] && D.p <= stls::kFusedMaxP) {
    const T *rows[4] = {pM.data(), pJ.data(), p2K.data(), pK.data()};
    for (int b = 0; b < 4; ++b)
      for (int w = 0; w < 2 * D.p + 1; ++w) A.int_3[b][w] = rows[b][static_cast<size_t>(A.lo[k]) * st + w];
  }
  int rc = upload(c, &A.pad_M[k], pM);
  if (!rc) rc = upload(c, &A.pad_K[k], pK);
  if (!rc) rc = upload(c, &A.pad_J[k], pJ);
  if (!rc) rc = upload(c, &A.pad_2K[k], p2K);
  return rc;
}

template <typename T>
int upload_padded_time(stls_ctx *c, AOps<T> &A, const stls::Dir1D &Tm, const std::vector<double> &bKt,
                       const std::vector<double> &bMt) {
  const int st = stls::band_row_stride(Tm.p, sizeof(T));
  const std::vector<T> pK = pad_band<T>(bKt, Tm.n, Tm.p, st, 1.0), pM = pad_band<T>(bMt, Tm.n, Tm.p, st, 1.0);
  const T *all[2] = {pK.data(), pM.data()};
  stls::toeplitz_rows<T>(all, 2, Tm.n, st, &A.lo_t, &A.hi_t);
  if (A.lo_t < A.hi_t && Tm.p <= stls::kFusedMaxP)
    for (int w = 0; w < 2 * Tm.p + 1; ++w) {
      A.int_Kt[w] = pK[static_cast<size_t>(A.lo_t) * st + w];
      A.int_Mt[w] = pM[static_cast<size_t>(A.lo_t) * st + w];
    }
  int rc = upload(c, &A.pad_Kt, pK);
  if (!rc) rc = upload(c, &A.pad_Mt, pM);
  return rc;
}

std::vector<double> transpose(const std::vector<double> &A, int n) {
  std::vector<double> T(A.size());
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) T[j * n + i] = A[i * n + j];
  return T;
}

// ---- timing ---------------------------------------------------------------------------
// Every phase is also an NVTX range of the same name (a no-op unless a
// profiler is attached); the whole create and solve calls are ranges too.
const char *const kPhaseName[5] = {"apply_A", "precond", "cg_vectors", "apply_A_f32", "apply_A_df"};

struct NvtxScope {
  explicit NvtxScope(const char *name) { nvtxRangePushA(name); }
  ~NvtxScope() { nvtxRangePop(); }
  NvtxScope(const NvtxScope &) = delete;
  NvtxScope &operator=(const NvtxScope &) = delete;
};

int phase_begin(stls_ctx *c, int phase) {
  nvtxRangePushA(kPhaseName[phase]);
  if (!c->timing) return -1;
  size_t idx = c->ev_pairs.size() * 2;
  while (c->ev_pool.size() < idx + 2) {
    cudaEvent_t ev;
    if (cudaEventCreate(&ev) != cudaSuccess) return -1;
    c->ev_pool.push_back(ev);
  }
  cudaEventRecord(c->ev_pool[idx], c->stream);
  c->ev_pairs.push_back({phase, static_cast<int>(idx)});
  return static_cast<int>(idx);
}

void phase_end(stls_ctx *c, int idx) {
  nvtxRangePop();
  if (idx < 0) return;
  cudaEventRecord(c->ev_pool[idx + 1], c->stream);
}

void collect_phases(stls_ctx *c) {
  for (auto &pr : c->ev_pairs) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->ev_pool[pr.second], c->ev_pool[pr.second + 1]) == cudaSuccess) {
      c->phase_ms[pr.first] += ms;
      c->phase_count[pr.first] += 1;
    }
  }
  c->ev_pairs.clear();
}

// ---- operators ------------------------------------------------------------------------
ModeView spatial_view(const stls_ctx *c, int k, long long outer_mult) {
  ModeView v{};
  v.n = c->n_s[k];
  long long inner = 1, outer = outer_mult;
  for (int l = 0; l < k; ++l) inner *= c->n_s[l];
  for (int l = k + 1; l < c->d; ++l) outer *= c->n_s[l];
  v.inner = inner;
  v.outer = outer;
  v.in_outer_stride = v.out_outer_stride = static_cast<long long>(v.n) * inner;
  return v;
}

// Spatial factors of Eq. A_kron on the cube, by the recurrence over modes
// k = 1..d of the partial Kronecker products
//   m  = M x ... x M,  j = sum (one J), k1 = sum (one K), kk = sum (two K's),
// so that M_s = m, L_s = k1 and J_s = j + 2 kk after the last mode.  The
// cross terms of J_s = int Lap B_i Lap B_j use int b''_i b_j = -K_ij on the
// Dirichlet basis, so int d_kk B_i d_ll B_j = (K_k x K_l x M ...) for k != l.
// X has `outer_mult` spatial slices.  Outputs (nullable): Ms, Js, Ls over all
// slices, and Ls_last over the last time slice only (A x needs it for W_t).
template <typename T>
int spatial_tree(stls_ctx *c, AOps<T> &A, const T *X, long long outer_mult, T *Ms, T *Js, T *Ls, T *Ls_last) {
  const int d = c->d, p = c->hs.prm.p_s;
  const T *cur[4] = {X, nullptr, nullptr, nullptr};  // m, j, k1, kk
  for (int k = 0; k < d - 1; ++k) {
    T **bank = A.abuf + (k % 2) * 4;
    stls::BandSpecT<T> s{};
    s.p = p;
    int slot_in[4] = {-1, -1, -1, -1};
    for (int a = 0; a < 4; ++a)
      if (cur[a] != nullptr) {
        slot_in[a] = s.n_in;
        s.in[s.n_in++] = cur[a];
      }
    const bool has_m = cur[0], has_j = cur[1], has_k1 = cur[2], has_kk = cur[3];
    int slot_out[4] = {-1, -1, -1, -1};
    const bool make[4] = {has_m, has_j || has_m, has_k1 || has_m, has_kk || has_k1};
    for (int a = 0; a < 4; ++a)
      if (make[a]) {
        slot_out[a] = s.n_out;
        s.out[s.n_out++] = bank[a];
      }
    auto add = [&](const T *band, int in_state, int out_state, T scale) {
      if (slot_in[in_state] < 0 || slot_out[out_state] < 0) return;
      s.term[s.n_terms++] = {band, slot_in[in_state], slot_out[out_state], scale};
    };
    add(A.band_M[k], 0, 0, T(1));
    add(A.band_M[k], 1, 1, T(1));
    add(A.band_J[k], 0, 1, T(1));
    add(A.band_M[k], 2, 2, T(1));
    add(A.band_K[k], 0, 2, T(1));
    add(A.band_M[k], 3, 3, T(1));
    add(A.band_K[k], 2, 3, T(1));
    STLS_LAUNCH(stls::launch_banded<T>(s, spatial_view(c, k, outer_mult), c->stream), "banded");
    for (int a = 0; a < 4; ++a) cur[a] = make[a] ? bank[a] : nullptr;
  }
  const int k = d - 1;
  {
    stls::BandSpecT<T> s{};
    s.p = p;
    int slot_in[4] = {-1, -1, -1, -1};
    for (int a = 0; a < 4; ++a)
      if (cur[a] != nullptr) {
        slot_in[a] = s.n_in;
        s.in[s.n_in++] = cur[a];
      }
    int o_ms = -1, o_js = -1, o_ls = -1;
    if (Ms) { o_ms = s.n_out; s.out[s.n_out++] = Ms; }
    if (Js) { o_js = s.n_out; s.out[s.n_out++] = Js; }
    if (Ls) { o_ls = s.n_out; s.out[s.n_out++] = Ls; }
    auto add = [&](const T *band, int in_state, int out_slot, T scale) {
      if (slot_in[in_state] < 0 || out_slot < 0) return;
      s.term[s.n_terms++] = {band, slot_in[in_state], out_slot, scale};
    };
    add(A.band_M[k], 0, o_ms, T(1));
    add(A.band_M[k], 1, o_js, T(1));
    add(A.band_M[k], 3, o_js, T(2));
    add(A.band_J[k], 0, o_js, T(1));
    add(A.band_K[k], 2, o_js, T(2));
    add(A.band_M[k], 2, o_ls, T(1));
    add(A.band_K[k], 0, o_ls, T(1));
    if (s.n_out > 0)
      STLS_LAUNCH(stls::launch_banded<T>(s, spatial_view(c, k, outer_mult), c->stream), "banded");
    if (Ls_last) {
      // L_s on the last time slice of every right-hand side
      stls::BandSpecT<T> t{};
      t.p = p;
      const long long off = static_cast<long long>(c->n_t - 1) * c->Ns;
      int sm_ = -1, sk1 = -1;
      t.in[t.n_in] = cur[0] + off;
      sm_ = t.n_in++;
      if (cur[2]) {
        t.in[t.n_in] = cur[2] + off;
        sk1 = t.n_in++;
      }
      t.out[t.n_out++] = Ls_last;
      t.term[t.n_terms++] = {A.band_K[k], sm_, 0, T(1)};
      if (sk1 >= 0) t.term[t.n_terms++] = {A.band_M[k], sk1, 0, T(1)};
      ModeView v = spatial_view(c, k, 1);
      v.outer = c->B;
      v.in_outer_stride = c->N;
      v.out_outer_stride = c->Ns;
      STLS_LAUNCH(stls::launch_banded<T>(t, v, c->stream), "banded");
    }
  }
  return STLS_OK;
}

bool is_geometry(const stls_ctx *c) { return c->hs.prm.geometry == 1; }

// Spatial factors of the least-squares matrix on the mapped cube (geometry =
// 1; weighted 1D factors M^w, K^w, J^w, E in the band arrays):
//   M_s = (x) M^w,  J_s = sum_k J^w_k + sum_{k != l} E_k (dir. k) E_l^T (dir. l),
//   L_s = sum_k K^w_k  (M^w in the other directions),
// by the recurrence over modes of the partial products m (all M^w), j (one
// J^w or a completed E / E^T pair), e (an E waiting for an E^T in a later
// direction) and f (an E^T waiting for an E): at every mode
//   m' = M m,  j' = M j + J m + E^T e + E f,  e' = M e + E m,  f' = M f + E^T m.
// L_s is needed on the last time slice only, by its own two-state recurrence
// (m, l' = M l + K m) on that slice.
int geometry_spatial(stls_ctx *c, AOps<double> &A, const double *X, double *Ms, double *Js, double *Ls_last) {
  const int d = c->d, p = c->hs.prm.p_s;
  const long long om = static_cast<long long>(c->B) * c->n_t;
  const double *cur[4] = {X, nullptr, nullptr, nullptr};  // m, j, e, f
  for (int k = 0; k < d; ++k) {
    const bool last = k == d - 1;
    double **bank = A.abuf + (k % 2) * 4;
    stls::BandSpecT<double> s{};
    s.p = p;
    int in[4] = {-1, -1, -1, -1};
    for (int a = 0; a < 4; ++a)
      if (cur[a] != nullptr) {
        in[a] = s.n_in;
        s.in[s.n_in++] = cur[a];
      }
    int out[4] = {-1, -1, -1, -1};
    if (last) {
      out[0] = s.n_out;
      s.out[s.n_out++] = Ms;
      out[1] = s.n_out;
      s.out[s.n_out++] = Js;
    } else {
      for (int a = 0; a < 4; ++a) {
        out[a] = s.n_out;
        s.out[s.n_out++] = bank[a];
      }
    }
    auto add = [&](const double *band, int from, int to) {
      if (in[from] < 0 || out[to] < 0) return;
      s.term[s.n_terms++] = {band, in[from], out[to], 1.0};
    };
    add(A.band_M[k], 0, 0);
    add(A.band_M[k], 1, 1);
    add(A.band_J[k], 0, 1);
    add(A.band_Et[k], 2, 1);
    add(A.band_E[k], 3, 1);
    add(A.band_M[k], 2, 2);
    add(A.band_E[k], 0, 2);
    add(A.band_M[k], 3, 3);
    add(A.band_Et[k], 0, 3);
    STLS_LAUNCH(stls::launch_banded<double>(s, spatial_view(c, k, om), c->stream), "banded (geometry)");
    if (!last)
      for (int a = 0; a < 4; ++a) cur[a] = bank[a];
  }
  if (Ls_last != nullptr) {
    // last time slice of every right-hand side: the first mode reads it from X
    // (stride N), later modes B x N_s buffers
    const double *lm = X + static_cast<long long>(c->n_t - 1) * c->Ns, *ll = nullptr;
    for (int k = 0; k < d; ++k) {
      const bool last = k == d - 1;
      stls::BandSpecT<double> s{};
      s.p = p;
      s.in[s.n_in++] = lm;
      if (ll) s.in[s.n_in++] = ll;
      double *om_ = c->lift_tmp[(k % 2) * 2], *ol = last ? Ls_last : c->lift_tmp[(k % 2) * 2 + 1];
      if (!last) s.out[s.n_out++] = om_;
      const int o_l = s.n_out;
      s.out[s.n_out++] = ol;
      if (!last) s.term[s.n_terms++] = {A.band_M[k], 0, 0, 1.0};
      s.term[s.n_terms++] = {A.band_K[k], 0, o_l, 1.0};
      if (ll) s.term[s.n_terms++] = {A.band_M[k], 1, o_l, 1.0};
      stls::ModeView v = spatial_view(c, k, 1);
      v.outer *= c->B;  // spatial_view(.., 1) covers one slice; B slices here
      v.in_outer_stride = v.out_outer_stride = static_cast<long long>(v.n) * v.inner;
      if (k == 0) {
        // inputs are slices of X: B right-hand sides N apart, outer index over (b, higher modes)
        v.outer = c->Ns / (static_cast<long long>(v.n) * v.inner);
        stls::ModeView vb = v;
        for (int b = 0; b < c->B; ++b) {
          stls::BandSpecT<double> sb = s;
          sb.in[0] = lm + static_cast<long long>(b) * c->N;
          for (int o = 0; o < sb.n_out; ++o) sb.out[o] = s.out[o] + static_cast<long long>(b) * c->Ns;
          STLS_LAUNCH(stls::launch_banded<double>(sb, vb, c->stream), "banded (geometry, L_s)");
        }
      } else {
        v.outer = static_cast<long long>(c->B) * (c->Ns / (static_cast<long long>(v.n) * v.inner));
        STLS_LAUNCH(stls::launch_banded<double>(s, v, c->stream), "banded (geometry, L_s)");
      }
      if (!last) {
        lm = om_;
        ll = ol;
      }
    }
  }
  return STLS_OK;
}

template <typename T>
stls::FusedA<T> fused_args(const stls_ctx *c, const AOps<T> &A) {
  stls::FusedA<T> f{};
  f.d = c->d;
  f.p_s = c->hs.prm.p_s;
  f.p_t = c->hs.prm.p_t;
  for (int k = 0; k < c->d; ++k) {
    f.n[k] = c->n_s[k];
    f.bM[k] = A.pad_M[k];
    f.bJ[k] = A.pad_J[k];
    f.bK[k] = A.pad_K[k];
    f.b2K[k] = A.pad_2K[k];
  }
  f.n_t = c->n_t;
  f.B = c->B;
  f.bKt = A.pad_Kt;
  f.bMt = A.pad_Mt;
  for (int k = 0; k < 3; ++k) {
    f.lo[k] = A.lo[k];
    f.hi[k] = A.hi[k];
  }
  f.lo_t = A.lo_t;
  f.hi_t = A.hi_t;
  for (int w = 0; w < 2 * stls::kFusedMaxP + 1; ++w) {
    f.iKt[w] = A.int_Kt[w];
    f.iMt[w] = A.int_Mt[w];
    for (int b = 0; b < 4; ++b) f.i3[b][w] = A.int_3[b][w];
  }
  for (int w = 0; w < 5; ++w) f.work[w] = A.abuf[w];
  f.ls_last = A.ls_buf;
  return f;
}

// y = A x in double-float arithmetic (refinement contexts with the fused A x):
// x, y are double-float images; the work buffers are those of the FP64 A x.
int apply_A_df_impl(stls_ctx *c, const stls::dfloat *x, stls::dfloat *y) {
  if (!c->have_df) return set_err(c, STLS_EINVAL, "double-float A x needs a refinement context with d = 2 or 3");
  const stls::FusedA<stls::dfloat> f = fused_args(c, c->adf);
  c->launches += c->d - 1;
  STLS_LAUNCH(stls::launch_fused_A<stls::dfloat>(f, x, y, c->stream), "fused A x (double-float)");
  return STLS_OK;
}

template <typename T>
int apply_A_impl(stls_ctx *c, AOps<T> &A, const T *x, T *y);

// q = A p in FP32 with the inner CG's step length fused into the last kernel
// ((p, q) and alpha = rz / (p, q) on st_in); falls back to the separate
// product when the fused A x does not apply.
int apply_A_f32_alpha(stls_ctx *c, const float *p, float *q) {
  if (stls::fused_A_supported(c->d, c->hs.prm.p_s, c->hs.prm.p_t)) {
    stls::FusedA<float> f = fused_args(c, c->a32);
    f.fuse = {p, c->st_in, c->alpha_partials, c->alpha_tickets};
    c->launches += c->d - 1;
    STLS_LAUNCH(stls::launch_fused_A<float>(f, p, q, c->stream), "fused A x (with alpha)");
    return STLS_OK;
  }
  int rc = apply_A_impl<float>(c, c->a32, p, q);
  if (rc) return rc;
  STLS_LAUNCH(stls::launch_cg_alpha<float>(p, q, c->N, c->B, c->st_in, c->rw, c->stream), "cg_alpha");
  return STLS_OK;
}

template <typename T>
int apply_A_impl(stls_ctx *c, AOps<T> &A, const T *x, T *y) {
  if constexpr (std::is_same_v<T, double>) {
    if (is_geometry(c)) {
      const int bank = (c->d - 1) % 2;
      T *Ms = A.abuf[bank * 4 + 0], *Js = A.abuf[bank * 4 + 1];
      int rc = geometry_spatial(c, A, x, Ms, Js, A.ls_buf);
      if (rc) return rc;
      stls::BandSpecT<T> s{};
      s.p = c->hs.prm.p_t;
      s.in[0] = Ms;
      s.in[1] = Js;
      s.n_in = 2;
      s.out[0] = y;
      s.n_out = 1;
      s.term[0] = {A.band_Kt, 0, 0, T(1)};
      s.term[1] = {A.band_Mt, 1, 0, T(1)};
      s.n_terms = 2;
      s.last_add = A.ls_buf;
      s.last_out = 0;
      ModeView v{};
      v.n = c->n_t;
      v.inner = c->Ns;
      v.outer = c->B;
      v.in_outer_stride = v.out_outer_stride = c->N;
      STLS_LAUNCH(stls::launch_banded<T>(s, v, c->stream), "banded(time)");
      return STLS_OK;
    }
  }
  if (stls::fused_A_supported(c->d, c->hs.prm.p_s, c->hs.prm.p_t)) {
    const stls::FusedA<T> f = fused_args(c, A);
    c->launches += c->d - 1;  // d launches in all
    STLS_LAUNCH(stls::launch_fused_A<T>(f, x, y, c->stream), "fused A x");
    return STLS_OK;
  }
  const int bank = (c->d - 1) % 2;
  T *Ms = A.abuf[bank * 4 + 0], *Js = A.abuf[bank * 4 + 1];
  int rc = spatial_tree<T>(c, A, x, static_cast<long long>(c->B) * c->n_t, Ms, Js, nullptr, A.ls_buf);
  if (rc) return rc;
  stls::BandSpecT<T> s{};
  s.p = c->hs.prm.p_t;
  s.in[0] = Ms;
  s.in[1] = Js;
  s.n_in = 2;
  s.out[0] = y;
  s.n_out = 1;
  s.term[0] = {A.band_Kt, 0, 0, T(1)};
  s.term[1] = {A.band_Mt, 1, 0, T(1)};
  s.n_terms = 2;
  s.last_add = A.ls_buf;  // W_t x L_s: W_t = e_{n_t} e_{n_t}^T touches the last time slice only
  s.last_out = 0;
  ModeView v{};
  v.n = c->n_t;
  v.inner = c->Ns;
  v.outer = c->B;
  v.in_outer_stride = v.out_outer_stride = c->N;
  STLS_LAUNCH(stls::launch_banded<T>(s, v, c->stream), "banded(time)");
  return STLS_OK;
}

ModeView fd_view(const stls_ctx *c, int k) {
  if (k < c->d) return spatial_view(c, k, static_cast<long long>(c->B) * c->n_t);
  ModeView v{};
  v.n = c->n_t;
  v.inner = c->Ns;
  v.outer = c->B;
  v.in_outer_stride = v.out_outer_stride = c->N;
  return v;
}

// Algorithm 1, steps 2-4: forward mode products with U_1^T..U_d^T, U_t^T, the
// division by lambda_t[i_t] + sum_k lambda_k[i_k] (fused into the last forward
// product), and backward mode products with U_1..U_d, U_t.
int fd_apply_impl(stls_ctx *c, const double *r, double *z) {
  if (c->hs.prm.precision != STLS_FP64) {
    c->launches += stls::tc_fd_launch_count(c->tc);
    cudaError_t e = stls::tc_fd_apply(c->tc, r, z, c->stream);
    if (e != cudaSuccess) return cuda_err(c, e, "tensor-core FD apply");
    return STLS_OK;
  }
  const int nprod = 2 * (c->d + 1);
  const double *src = r;
  if (c->geo_dinv != nullptr) {  // P^G = D^{1/2} Pbar^G D^{1/2}: (P^G)^{-1} r = D^{-1/2} Pbar^{-1} D^{-1/2} r
    STLS_LAUNCH(stls::launch_scale(r, c->geo_dinv, c->geo_tmp, c->N, c->B, c->stream), "scale");
    src = c->geo_tmp;
  }
  for (int s = 0; s < nprod; ++s) {
    const bool fwd = s <= c->d;
    const int k = fwd ? s : s - c->d - 1;
    double *dst = (s == nprod - 1) ? z : c->fd_tmp[s % 2];
    const bool divide = fwd && k == c->d;
    STLS_LAUNCH(stls::launch_modeprod_f64(src, dst, fwd ? c->Uf[k] : c->Ub[k], fd_view(c, k),
                                          divide ? c->lam_t : nullptr, divide ? c->lam_s : nullptr,
                                          c->stream),
                "modeprod");
    src = dst;
  }
  if (c->geo_dinv != nullptr)
    STLS_LAUNCH(stls::launch_scale(z, c->geo_dinv, z, c->N, c->B, c->stream), "scale");
  return STLS_OK;
}

// lambda_s[c] = sum_k lambda_k[i_k(c)] over the colexicographic spatial index
std::vector<double> spatial_eigenvalue_sums(const stls_ctx *c) {
  std::vector<double> ls(c->Ns, 0.0);
  for (long long idx = 0; idx < c->Ns; ++idx) {
    long long rem = idx;
    double s = 0.0;
    for (int k = 0; k < c->d; ++k) {
      s += c->hs.eig_s[k].lam[rem % c->n_s[k]];
      rem /= c->n_s[k];
    }
    ls[idx] = s;
  }
  return ls;
}

// D^{-1/2} of P^G = D^{1/2} Pbar^G D^{1/2}, D = diag(A) / diag(Pbar^G) over the
// colexicographic index (Sec. 4.4), from the diagonals of the 1D factors:
//   diag(A) = Kt x Mw_s + Mt x (sum_k Jw_k + sum_{k != l} E_k E_l) + Wt x sum_k Kw_k,
//   diag(Pbar^G) = Kg_t x Mg_s + Mg_t x sum_k Jg_k   (M in the other directions).
std::vector<double> geometry_scaling(const stls_ctx *c) {
  const stls::HostSetup &hs = c->hs;
  const int d = c->d, nt = c->n_t;
  auto diag = [](const std::vector<double> &A, int n) {
    std::vector<double> v(n);
    for (int i = 0; i < n; ++i) v[i] = A[static_cast<size_t>(i) * n + i];
    return v;
  };
  std::vector<std::vector<double>> dMw(d), dKw(d), dJw(d), dE(d), dMg(d), dJg(d);
  for (int k = 0; k < d; ++k) {
    const int n = c->n_s[k];
    dMw[k] = diag(hs.geo[k].M, n);
    dKw[k] = diag(hs.geo[k].K, n);
    dJw[k] = diag(hs.geo[k].J, n);
    dE[k] = diag(hs.geo[k].E, n);
    dMg[k] = diag(hs.pg_M[k], n);
    dJg[k] = diag(hs.pg_J[k], n);
  }
  const std::vector<double> dKt = diag(hs.time.K, nt), dMt = diag(hs.time.M, nt);
  const std::vector<double> dKgt = diag(hs.pg_Kt, nt), dMgt = diag(hs.pg_Mt, nt);
  std::vector<double> out(c->N);
  std::vector<int> idx(d);
  for (long long sidx = 0; sidx < c->Ns; ++sidx) {
    long long rem = sidx;
    for (int k = 0; k < d; ++k) {
      idx[k] = static_cast<int>(rem % c->n_s[k]);
      rem /= c->n_s[k];
    }
    double ms = 1.0, mg = 1.0;
    for (int k = 0; k < d; ++k) {
      ms *= dMw[k][idx[k]];
      mg *= dMg[k][idx[k]];
    }
    double js = 0.0, ls = 0.0, jg = 0.0;
    for (int k = 0; k < d; ++k) {
      double tj = dJw[k][idx[k]], tl = dKw[k][idx[k]], tg = dJg[k][idx[k]];
      for (int l = 0; l < d; ++l)
        if (l != k) {
          tj *= dMw[l][idx[l]];
          tl *= dMw[l][idx[l]];
          tg *= dMg[l][idx[l]];
        }
      js += tj;
      ls += tl;
      jg += tg;
      for (int l = 0; l < d; ++l) {
        if (l == k) continue;
        double te = dE[k][idx[k]] * dE[l][idx[l]];
        for (int m = 0; m < d; ++m)
          if (m != k && m != l) te *= dMw[m][idx[m]];
        js += te;
      }
    }
    for (int t = 0; t < nt; ++t) {
      const double a = dKt[t] * ms + dMt[t] * js + (t == nt - 1 ? hs.time.end_values[t] * hs.time.end_values[t] : 0.0) * ls;
      const double pg = dKgt[t] * mg + dMgt[t] * jg;
      out[static_cast<size_t>(t) * c->Ns + sidx] = 1.0 / std::sqrt(a / pg);
    }
  }
  return out;
}

// Residual history: after every read of the solver state, entry `iters` of
// right-hand side b holds its latest relative residual (a new entry per
// iteration or outer step; a recomputed residual overwrites its entry).
constexpr int kMaxHistory = 1 << 20;
void history_reset(stls_ctx *c) { c->hist.assign(c->B, std::vector<double>(1, 1.0)); }
void history_record(stls_ctx *c) {
  for (int b = 0; b < c->B && b < static_cast<int>(c->hist.size()); ++b) {
    const CGState &s = c->st_host[b];
    if (s.iters < 0 || s.iters >= kMaxHistory) continue;
    std::vector<double> &h = c->hist[b];
    if (static_cast<int>(h.size()) < s.iters + 1) h.resize(s.iters + 1, s.rel_res);
    h[s.iters] = s.rel_res;
    if (!(s.nF2 > 0.0)) h[0] = 0.0;  // F = 0: u = 0 with a zero residual
  }
}

int check_ptr(stls_ctx *c, const void *ptr, const char *name) {
  if (ptr == nullptr || (reinterpret_cast<uintptr_t>(ptr) & 7u) != 0)
    return set_err(c, STLS_EINVAL, std::string(name) + " is NULL or not 8-byte aligned");
  return STLS_OK;
}

int solve_impl(stls_ctx *c, const double *F, double *u, double tol, int maxit, stls_solve_info *info) {
  if (!(tol >= 0.0) || maxit < 0) return set_err(c, STLS_EINVAL, "tol must be >= 0 and maxit >= 0");
  if (check_ptr(c, F, "F") || check_ptr(c, u, "u")) return STLS_EINVAL;
  const long long N = c->N;
  const int B = c->B;
  const int flex = c->hs.prm.flexible;
  history_reset(c);
  int ph = phase_begin(c, 2);
  STLS_LAUNCH(stls::launch_cg_init(F, u, c->r, N, B, c->st, c->rw, c->stream), "cg_init");
  phase_end(c, ph);
  ph = phase_begin(c, 1);
  int rc = fd_apply_impl(c, c->r, c->z);
  if (rc) return rc;
  phase_end(c, ph);
  ph = phase_begin(c, 2);
  STLS_LAUNCH(stls::launch_cg_beta(c->z, c->r, c->q, N, B, flex, 1, c->st, c->rw, c->stream), "cg_beta");
  STLS_LAUNCH(stls::launch_cg_p(c->z, c->p, N, B, 1, c->st, c->stream), "cg_p");
  phase_end(c, ph);
  for (int it = 1; it <= maxit; ++it) {
    ph = phase_begin(c, 0);
    rc = apply_A_impl<double>(c, c->a64, c->p, c->q);
    if (rc) return rc;
    phase_end(c, ph);
    ph = phase_begin(c, 2);
    STLS_LAUNCH(stls::launch_cg_alpha(c->p, c->q, N, B, c->st, c->rw, c->stream), "cg_alpha");
    STLS_LAUNCH(stls::launch_cg_xr(u, c->r, c->p, c->q, N, B, tol, c->st, c->rw, c->stream), "cg_xr");
    phase_end(c, ph);
    STLS_CK(cudaMemcpyAsync(c->st_host, c->st, sizeof(CGState) * B, cudaMemcpyDeviceToHost, c->stream),
            "state copy");
    STLS_CK(cudaStreamSynchronize(c->stream), "sync");
    history_record(c);
    if (c->hs.prm.precision != STLS_FP64 && stls::tc_fd_error(c->tc))
      return set_err(c, STLS_ECUDA, "tensor-core FD apply: a bounded mbarrier wait timed out");
    bool any = false;
    for (int b = 0; b < B; ++b) any = any || c->st_host[b].active;
    if (!any) break;
    ph = phase_begin(c, 1);
    rc = fd_apply_impl(c, c->r, c->z);
    if (rc) return rc;
    phase_end(c, ph);
    ph = phase_begin(c, 2);
    STLS_LAUNCH(stls::launch_cg_beta(c->z, c->r, c->q, N, B, flex, 0, c->st, c->rw, c->stream), "cg_beta");
    STLS_LAUNCH(stls::launch_cg_p(c->z, c->p, N, B, 0, c->st, c->stream), "cg_p");
    phase_end(c, ph);
  }
  // true FP64 residual ||F - A u|| at exit
  rc = apply_A_impl<double>(c, c->a64, u, c->q);
  if (rc) return rc;
  STLS_LAUNCH(stls::launch_true_residual(F, c->q, N, B, c->st, c->rw, c->stream), "true_residual");
  STLS_CK(cudaMemcpyAsync(c->st_host, c->st, sizeof(CGState) * B, cudaMemcpyDeviceToHost, c->stream),
          "state copy");
  STLS_CK(cudaStreamSynchronize(c->stream), "sync");
  history_record(c);
  if (c->timing) collect_phases(c);
  int first_bad = STLS_OK;
  for (int b = 0; b < B; ++b) {
    const CGState &s = c->st_host[b];
    int status = s.status;
    if (status == STLS_OK && s.active) status = STLS_ENOTCONV;
    if (info != nullptr) {
      info[b].iters = s.iters;
      info[b].status = status;
      info[b].rel_res = s.rel_res;
      info[b].true_rel_res = s.nF2 > 0 ? std::sqrt(s.true_rr / s.nF2) : 0.0;
      info[b].outer = 0;
      info[b].outer_df = 0;
    }
    if (status != STLS_OK && first_bad == STLS_OK) first_bad = status;
  }
  if (first_bad != STLS_OK) {
    static const char *names[] = {"ok", "einval", "enomem", "ecuda", "not converged", "breakdown",
                                  "non-finite value"};
    set_err(c, first_bad, std::string("solve: ") + names[first_bad]);
  }
  return first_bad;
}

// Iterative refinement (mixed forms, refine = 1).  Outer loop in FP64:
// r = F - A u (FP64 A x; provisional steps in double-float), stop when
// ||r|| / ||F|| <= tol; otherwise solve A d = r 2^-k (||r|| = f 2^k, f in
// [0.5, 1): an exact scaling) approximately by flexible CG in FP32 (FP32
// vectors and A p, the tensor-core preconditioner, inner products compensated
// in FP32 per thread and summed in FP64) until its residual falls below the
// inner tolerance, and update u += 2^k d in FP64.
// One step of the inner flexible CG of the refinement form, as the body of a
// graph while loop: z = P r, beta and p (first step: st.iters == 0, read on
// the device), q = A p with alpha, then x, r and the loop condition.  The
// inner tolerance comes from the state (ir_start wrote it).
int inner_graph_body(stls_ctx *c, float *rpad, int pad_n0, int pad_np0, cudaGraphConditionalHandle h) {
  const long long N = c->N;
  const int B = c->B;
  if (rpad != nullptr) {
    c->launches += stls::tc_fd_launch_count(c->tc) - 1;
    STLS_CK(stls::tc_fd_apply_f32_padded(c->tc, c->zi, c->stream), "tensor-core FD apply");
  } else {
    c->launches += stls::tc_fd_launch_count(c->tc);
    STLS_CK(stls::tc_fd_apply_f32(c->tc, c->ri, c->zi, c->stream), "tensor-core FD apply");
  }
  STLS_LAUNCH(stls::launch_cg_beta<float>(c->zi, c->ri, c->qi, N, B, 1, -1, c->st_in, c->rw, c->stream),
              "cg_beta");
  STLS_LAUNCH(stls::launch_cg_p<float>(c->zi, c->pi, N, B, -1, c->st_in, c->stream,
                                       rpad != nullptr ? c->di : nullptr, c->rw.tickets),
              "cg_p");
  const int rc = apply_A_f32_alpha(c, c->pi, c->qi);
  if (rc) return rc;
  if (rpad != nullptr)
    STLS_LAUNCH(stls::launch_cg_xr_pad(c->di, c->ri, c->pi, c->qi, N, B, -1.0, c->st_in, c->rw, rpad, pad_n0,
                                       pad_np0, 1, c->stream),
                "cg_xr");
  else
    STLS_LAUNCH(stls::launch_cg_xr<float>(c->di, c->ri, c->pi, c->qi, N, B, -1.0, c->st_in, c->rw, c->stream),
                "cg_xr");
  STLS_LAUNCH(stls::launch_inner_cond(c->st_in, B, stls::tc_fd_error_flag(c->tc), h, c->stream), "inner_cond");
  return STLS_OK;
}

// Builds the inner-loop graph (a while node around inner_graph_body, captured
// on a private stream).  Returns false, and marks the context, when the graph
// cannot be built: the solve then drives the loop from the host.
bool build_inner_graph(stls_ctx *c, float *rpad, int pad_n0, int pad_np0) {
  cudaGraph_t g = nullptr;
  cudaGraphConditionalHandle h = 0;
  cudaStream_t cap = nullptr;
  bool ok = cudaGraphCreate(&g, 0) == cudaSuccess &&
            cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) == cudaSuccess &&
            cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) == cudaSuccess;
  cudaGraphNodeParams cp = {};
  cudaGraphNode_t node = nullptr;
  if (ok) {
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    ok = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp) == cudaSuccess;
  }
  if (ok) {
    cudaStream_t user = c->stream;
    const long long l0 = c->launches;
    c->stream = cap;
    if (cudaStreamBeginCaptureToGraph(cap, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      const int rc = inner_graph_body(c, rpad, pad_n0, pad_np0, h);
      cudaGraph_t body = nullptr;
      ok = cudaStreamEndCapture(cap, &body) == cudaSuccess && rc == STLS_OK;
    } else {
      ok = false;
    }
    c->stream = user;
    c->ig_body_launches = c->launches - l0;
    c->launches = l0;
  }
  if (ok) ok = cudaGraphInstantiate(&c->ig_exec, g, 0) == cudaSuccess;
  if (cap != nullptr) cudaStreamDestroy(cap);
  if (!ok) {
    if (g != nullptr) cudaGraphDestroy(g);
    c->ig_exec = nullptr;
    c->ig_failed = true;
    cudaGetLastError();  // clear the failed calls' error state
    c->err.clear();
    return false;
  }
  c->ig_graph = g;
  return true;
}

// u_host_early != NULL (stls_solve_host): before each FP64 residual, u (final
// unless that residual asks for another step) is copied to u_host_early on
// c->copy_stream, overlapping the FP64 A x; c->early_final tells whether the
// last copy holds the returned u.
int solve_ir_impl(stls_ctx *c, const double *F, double *u, double tol, int maxit, stls_solve_info *info,
                  double *u_host_early = nullptr) {
  if (!(tol >= 0.0) || maxit < 0) return set_err(c, STLS_EINVAL, "tol must be >= 0 and maxit >= 0");
  if (check_ptr(c, F, "F") || check_ptr(c, u, "u")) return STLS_EINVAL;
  const long long N = c->N;
  const int B = c->B;
  // Inner target: fixed inner_tol when given.  Otherwise: one outer step
  // reduces the FP64 residual by about max(eta, 4e-4) (the FP32 inner operator
  // bounds the contraction), so the reduction R = tol / (||r|| / ||F||) still
  // needed by the worst right-hand side is split evenly over the
  // K = ceil(log R / log 1e-3) steps it takes: eta = R^(1/K), at least 1e-4.
  // A cap on inner iterations per outer step stops an inner solve that
  // stagnates; the FP64 outer residual decides convergence.
  const bool adaptive = !(c->hs.prm.inner_tol > 0.0);
  const double eta_fixed = c->hs.prm.inner_tol, eta_min = 1e-4, kStep = 1e-3;
  const int kMaxOuter = 100, kMaxInnerPerOuter = 400;
  double *r64 = c->r, *q64 = c->q;
  history_reset(c);
  int ph = phase_begin(c, 2);
  STLS_LAUNCH(stls::launch_cg_init(F, u, r64, N, B, c->st, c->rw, c->stream), "cg_init");
  phase_end(c, ph);
  // Provisional residuals: an outer step whose predicted residual is far
  // above both tol and the accuracy of double-float arithmetic takes F - A u
  // with the double-float A x (FP32 operations only); the FP64 residual
  // confirms every convergence test, a non-finite norm and the last step.
  // The prediction is ||r|| max(inner residual reached, 4e-4).
  const double kDfMargin = 100.0, kDfFloor = 1e-8, kContractFloor = 4e-4;
  double *xdf_buf = c->p;  // FP64 CG vectors, unused by the refinement form
  auto fp64_residual = [&](int count) -> int {
    if (u_host_early != nullptr && !c->early_final) {
      STLS_CK(cudaEventRecord(c->ev_u, c->stream), "event");
      STLS_CK(cudaStreamWaitEvent(c->copy_stream, c->ev_u, 0), "event wait");
      STLS_CK(cudaMemcpyAsync(u_host_early, u, sizeof(double) * static_cast<size_t>(B) * N, cudaMemcpyDeviceToHost,
                              c->copy_stream),
              "D2H copy of u");
      STLS_CK(cudaEventRecord(c->ev_copied, c->copy_stream), "event");
      c->early_issued = c->early_final = true;
    }
    int ph2 = phase_begin(c, 0);
    int rc2 = apply_A_impl<double>(c, c->a64, u, q64);
    if (rc2) return rc2;
    phase_end(c, ph2);
    ph2 = phase_begin(c, 2);
    STLS_LAUNCH(stls::launch_ir_residual(F, q64, r64, N, B, tol, count, c->st, c->rw, c->stream), "ir_residual");
    phase_end(c, ph2);
    return STLS_OK;
  };
  auto read_state = [&]() -> int {
    STLS_CK(cudaMemcpyAsync(c->st_host, c->st, sizeof(CGState) * B, cudaMemcpyDeviceToHost, c->stream),
            "state copy");
    STLS_CK(cudaStreamSynchronize(c->stream), "sync");
    history_record(c);
    return STLS_OK;
  };
  std::vector<CGState> inner_host(B);
  int total_inner = 0, outer = 0, rc = STLS_OK;
  bool last_df = false;
  int pad_n0 = 0, pad_np0 = 0;
  float *rpad = stls::tc_fd_padded_input(c->tc, &pad_n0, &pad_np0);
  for (; outer < kMaxOuter; ++outer) {
    rc = read_state();
    if (rc) return rc;
    if (last_df) {
      bool confirm = total_inner >= maxit || outer + 1 >= kMaxOuter;
      for (int b = 0; b < B; ++b)
        if (c->st_host[b].active && !(c->st_host[b].rel_res > tol && std::isfinite(c->st_host[b].rel_res)))
          confirm = true;
      if (confirm) {
        rc = fp64_residual(0);
        if (!rc) rc = read_state();
        if (rc) return rc;
        last_df = false;
      }
    }
    bool any = false;
    double worst = 0.0;
    for (int b = 0; b < B; ++b)
      if (c->st_host[b].active) {
        any = true;
        worst = std::max(worst, c->st_host[b].rel_res);
      }
    if (!any || total_inner >= maxit) break;
    double eta = eta_fixed;
    if (adaptive) {
      const double R = (worst > 0.0 && tol > 0.0) ? std::min(1.0, tol / worst) : 0.0;
      if (R <= 0.0) {
        eta = eta_min;
      } else {
        const int K = std::max(1, static_cast<int>(std::ceil(std::log(R) / std::log(kStep) - 1e-9)));
        eta = std::min(0.1, std::max(eta_min, std::pow(R, 1.0 / K)));
      }
    }
    // ---- inner flexible CG in FP32 on A d = r 2^-k ----
    ph = phase_begin(c, 2);
    const int budget = std::min(maxit - total_inner, kMaxInnerPerOuter);
    STLS_LAUNCH(stls::launch_ir_start(r64, c->ri, c->di, N, B, c->st, c->st_in, c->rw, rpad, pad_n0, pad_np0, eta,
                                      budget, c->stream),
                "ir_start");
    phase_end(c, ph);
    // The inner loop runs as one graph launch (no host round trip per step)
    // unless phases are being timed or the graph could not be built.
    const bool graph = !c->timing && !c->ig_failed &&
                       (c->ig_exec != nullptr || build_inner_graph(c, rpad, pad_n0, pad_np0));
    if (graph) {
      STLS_CK(cudaGraphLaunch(c->ig_exec, c->stream), "inner CG graph");
    } else {
      ph = phase_begin(c, 1);
      if (rpad != nullptr) {  // ir_start wrote r into the preconditioner's input rows
        c->launches += stls::tc_fd_launch_count(c->tc) - 1;
        STLS_CK(stls::tc_fd_apply_f32_padded(c->tc, c->zi, c->stream), "tensor-core FD apply");
      } else {
        c->launches += stls::tc_fd_launch_count(c->tc);
        STLS_CK(stls::tc_fd_apply_f32(c->tc, c->ri, c->zi, c->stream), "tensor-core FD apply");
      }
      phase_end(c, ph);
      ph = phase_begin(c, 2);
      STLS_LAUNCH(stls::launch_cg_beta<float>(c->zi, c->ri, c->qi, N, B, 1, 1, c->st_in, c->rw, c->stream),
                  "cg_beta");
      STLS_LAUNCH(stls::launch_cg_p<float>(c->zi, c->pi, N, B, 1, c->st_in, c->stream), "cg_p");
      phase_end(c, ph);
      for (int it = 1; it <= budget; ++it) {
        ph = phase_begin(c, 3);
        rc = apply_A_f32_alpha(c, c->pi, c->qi);  // q = A p and alpha
        if (rc) return rc;
        phase_end(c, ph);
        ph = phase_begin(c, 2);
        if (rpad != nullptr)  // r also goes straight into the TF32 preconditioner's input rows; d += a p deferred
          STLS_LAUNCH(stls::launch_cg_xr_pad(c->di, c->ri, c->pi, c->qi, N, B, eta, c->st_in, c->rw, rpad, pad_n0,
                                             pad_np0, 1, c->stream),
                      "cg_xr");
        else
          STLS_LAUNCH(stls::launch_cg_xr<float>(c->di, c->ri, c->pi, c->qi, N, B, eta, c->st_in, c->rw, c->stream),
                      "cg_xr");
        phase_end(c, ph);
        STLS_CK(cudaMemcpyAsync(inner_host.data(), c->st_in, sizeof(CGState) * B, cudaMemcpyDeviceToHost,
                                c->stream),
                "state copy");
        STLS_CK(cudaStreamSynchronize(c->stream), "sync");
        if (stls::tc_fd_error(c->tc))
          return set_err(c, STLS_ECUDA, "tensor-core FD apply: a bounded mbarrier wait timed out");
        bool inner_any = false;
        for (int b = 0; b < B; ++b) inner_any = inner_any || inner_host[b].active;
        if (!inner_any) break;
        ph = phase_begin(c, 1);
        if (rpad != nullptr) {
          c->launches += stls::tc_fd_launch_count(c->tc) - 1;  // no padding pass
          STLS_CK(stls::tc_fd_apply_f32_padded(c->tc, c->zi, c->stream), "tensor-core FD apply");
        } else {
          c->launches += stls::tc_fd_launch_count(c->tc);
          STLS_CK(stls::tc_fd_apply_f32(c->tc, c->ri, c->zi, c->stream), "tensor-core FD apply");
        }
        phase_end(c, ph);
        ph = phase_begin(c, 2);
        STLS_LAUNCH(stls::launch_cg_beta<float>(c->zi, c->ri, c->qi, N, B, 1, 0, c->st_in, c->rw, c->stream),
                    "cg_beta");
        STLS_LAUNCH(stls::launch_cg_p<float>(c->zi, c->pi, N, B, 0, c->st_in, c->stream,
                                             rpad != nullptr ? c->di : nullptr, c->rw.tickets),
                    "cg_p");
        phase_end(c, ph);
      }
    }
    if (graph) {  // the inner states after the loop, and the kernels it ran
      STLS_CK(cudaMemcpyAsync(inner_host.data(), c->st_in, sizeof(CGState) * B, cudaMemcpyDeviceToHost,
                              c->stream),
              "state copy");
      STLS_CK(cudaStreamSynchronize(c->stream), "sync");
      if (stls::tc_fd_error(c->tc))
        return set_err(c, STLS_ECUDA, "tensor-core FD apply: a bounded mbarrier wait timed out");
      int steps = 1;
      for (int b = 0; b < B; ++b) steps = std::max(steps, inner_host[b].iters);
      c->launches += c->ig_body_launches * steps;
    }
    int its = 0;
    double inner_worst = 0.0;
    for (int b = 0; b < B; ++b) {
      its = std::max(its, inner_host[b].iters);
      if (c->st_host[b].active) inner_worst = std::max(inner_worst, inner_host[b].rel_res);
    }
    total_inner += std::max(its, 1);
    // ---- FP64 correction and residual ----
    const double predicted = worst * std::max(inner_worst, kContractFloor);
    const bool use_df = c->have_df && predicted > kDfMargin * tol && predicted > kDfFloor && total_inner < maxit;
    stls::dfloat *xdf = reinterpret_cast<stls::dfloat *>(xdf_buf), *ydf = reinterpret_cast<stls::dfloat *>(q64);
    ph = phase_begin(c, 2);
    // (with rpad the last CG updates deferred d += alpha p: the correction applies it)
    STLS_LAUNCH(stls::launch_ir_correct(u, c->di, rpad != nullptr ? c->pi : nullptr, c->st_in,
                                        use_df ? xdf : nullptr, N, B, c->st, c->stream),
                "ir_correct");
    c->early_final = false;  // u changed since any earlier copy
    phase_end(c, ph);
    if (use_df) {  // the correction kernel wrote the double-float image of u
      ph = phase_begin(c, 4);
      rc = apply_A_df_impl(c, xdf, ydf);
      if (rc) return rc;
      phase_end(c, ph);
      ph = phase_begin(c, 2);
      STLS_LAUNCH(stls::launch_ir_residual_df(F, ydf, r64, N, B, c->st, c->rw, c->stream), "ir_residual_df");
      phase_end(c, ph);
      last_df = true;
    } else {
      rc = fp64_residual(1);
      if (rc) return rc;
      last_df = false;
    }
  }
  if (last_df) {  // the outer step limit ended the loop after a provisional residual
    rc = fp64_residual(0);
    if (rc) return rc;
  }
  STLS_CK(cudaMemcpyAsync(c->st_host, c->st, sizeof(CGState) * B, cudaMemcpyDeviceToHost, c->stream),
          "state copy");
  STLS_CK(cudaStreamSynchronize(c->stream), "sync");
  history_record(c);
  if (c->timing) collect_phases(c);
  int first_bad = STLS_OK;
  for (int b = 0; b < B; ++b) {
    const CGState &s = c->st_host[b];
    int status = s.status;
    if (status == STLS_OK && s.active) status = STLS_ENOTCONV;
    if (info != nullptr) {
      info[b].iters = total_inner;
      info[b].status = status;
      info[b].rel_res = s.rel_res;
      info[b].true_rel_res = s.nF2 > 0 ? std::sqrt(s.rr / s.nF2) : 0.0;
      info[b].outer = s.iters;
      info[b].outer_df = s.df_iters;
    }
    if (status != STLS_OK && first_bad == STLS_OK) first_bad = status;
  }
  if (first_bad != STLS_OK) {
    static const char *names[] = {"ok", "einval", "enomem", "ecuda", "not converged", "breakdown",
                                  "non-finite value"};
    set_err(c, first_bad, std::string("solve (refinement): ") + names[first_bad]);
  }
  return first_bad;
}

}  // namespace

namespace stls {
// Error text for context-free calls, read back with stls_last_error(NULL).
void set_thread_error(const std::string &msg) { g_create_error = msg; }
}  // namespace stls

// ---- C ABI ----------------------------------------------------------------------------
extern "C" {

const char *stls_last_error(const stls_ctx *ctx) {
  return ctx == nullptr ? g_create_error.c_str() : ctx->err.c_str();
}

void stls_destroy(stls_ctx *ctx) {
  if (ctx == nullptr) return;
  cudaStreamSynchronize(ctx->stream);
  if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
  if (ctx->ev_u) cudaEventDestroy(ctx->ev_u);
  if (ctx->ev_copied) cudaEventDestroy(ctx->ev_copied);
  if (ctx->ig_exec) cudaGraphExecDestroy(ctx->ig_exec);
  if (ctx->ig_graph) cudaGraphDestroy(ctx->ig_graph);
  stls::tc_fd_destroy(ctx->tc);
  for (void *v : ctx->allocations) cudaFree(v);
  if (ctx->st_host) cudaFreeHost(ctx->st_host);
  for (cudaEvent_t ev : ctx->ev_pool) cudaEventDestroy(ev);
  delete ctx;
}

int stls_create(stls_ctx **out, const stls_params *prm, void *cuda_stream) {
  NvtxScope range("stls_create");
  g_create_error.clear();
  if (out == nullptr || prm == nullptr) {
    g_create_error = "out and prm must not be NULL";
    return STLS_EINVAL;
  }
  *out = nullptr;
  stls_ctx *c = new stls_ctx();
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  std::string err;
  if (!stls::build_setup(*prm, c->hs, err)) {
    g_create_error = err;
    delete c;
    return STLS_EINVAL;
  }
  const stls_params &P = c->hs.prm;
  c->d = P.d;
  c->B = P.batch;
  c->n_t = c->hs.time.n;
  c->Ns = 1;
  for (int k = 0; k < c->d; ++k) {
    c->n_s[k] = c->hs.space[k].n;
    c->Ns *= c->n_s[k];
  }
  c->N = c->Ns * c->n_t;
  auto fail = [&](int code) {
    g_create_error = c->err;
    stls_destroy(c);
    return code;
  };
  int rc = STLS_OK;
  const bool refine = P.refine != 0;
  // double-float A x for the provisional outer residuals of the refinement form
  const bool df = refine && P.fp64_residuals == 0 && stls::fused_A_supported(c->d, P.p_s, P.p_t);
  c->have_df = df;
  auto to_f32 = [](const std::vector<double> &v) { return std::vector<float>(v.begin(), v.end()); };
  const bool geo = P.geometry == 1;
  for (int k = 0; k < c->d && !rc; ++k) {
    const stls::Dir1D &D = c->hs.space[k];
    // the mapped cube's A uses the weighted factors (E and E^T for the cross terms)
    const std::vector<double> &mM = geo ? c->hs.geo[k].M : D.M, &mK = geo ? c->hs.geo[k].K : D.K,
                              &mJ = geo ? c->hs.geo[k].J : D.J;
    const std::vector<double> bM = stls::to_band(mM, D.n, D.p), bK = stls::to_band(mK, D.n, D.p),
                              bJ = stls::to_band(mJ, D.n, D.p);
    if (geo) {
      rc = upload(c, &c->a64.band_E[k], stls::to_band(c->hs.geo[k].E, D.n, D.p));
      if (!rc) rc = upload(c, &c->a64.band_Et[k], stls::to_band(transpose(c->hs.geo[k].E, D.n), D.n, D.p));
      if (rc) break;
    }
    rc = upload(c, &c->a64.band_M[k], bM);
    if (!rc) rc = upload(c, &c->a64.band_K[k], bK);
    if (!rc) rc = upload(c, &c->a64.band_J[k], bJ);
    if (!rc && refine) rc = upload(c, &c->a32.band_M[k], to_f32(bM));
    if (!rc && refine) rc = upload(c, &c->a32.band_K[k], to_f32(bK));
    if (!rc && refine) rc = upload(c, &c->a32.band_J[k], to_f32(bJ));
    if (!rc) rc = upload_padded(c, c->a64, k, D, bM, bK, bJ);
    if (!rc && refine) rc = upload_padded(c, c->a32, k, D, bM, bK, bJ);
    if (!rc && df) rc = upload_padded(c, c->adf, k, D, bM, bK, bJ);
    if (!rc) rc = upload(c, &c->Uf[k], transpose(c->hs.eig_s[k].U, D.n));
    if (!rc) rc = upload(c, &c->Ub[k], c->hs.eig_s[k].U);
  }
  const stls::Dir1D &Tm = c->hs.time;
  {
    const std::vector<double> bKt = stls::to_band(Tm.K, Tm.n, Tm.p), bMt = stls::to_band(Tm.M, Tm.n, Tm.p);
    if (!rc) rc = upload(c, &c->a64.band_Kt, bKt);
    if (!rc) rc = upload(c, &c->a64.band_Mt, bMt);
    if (!rc && refine) rc = upload(c, &c->a32.band_Kt, to_f32(bKt));
    if (!rc && refine) rc = upload(c, &c->a32.band_Mt, to_f32(bMt));
    if (!rc) rc = upload_padded_time(c, c->a64, Tm, bKt, bMt);
    if (!rc && refine) rc = upload_padded_time(c, c->a32, Tm, bKt, bMt);
    if (!rc && df) rc = upload_padded_time(c, c->adf, Tm, bKt, bMt);
  }
  if (!rc) rc = upload(c, &c->Uf[c->d], transpose(c->hs.eig_t.U, Tm.n));
  if (!rc) rc = upload(c, &c->Ub[c->d], c->hs.eig_t.U);
  if (!rc) rc = upload(c, &c->lam_t, c->hs.eig_t.lam);
  if (!rc) rc = upload(c, &c->e_end, Tm.end_values);
  if (!rc) rc = upload(c, &c->m_int, Tm.integrals);
  if (!rc) rc = upload(c, &c->ones_t, std::vector<double>(Tm.n, 1.0));
  if (!rc) rc = upload(c, &c->zeros_t, std::vector<double>(Tm.n, 0.0));
  if (!rc) rc = upload(c, &c->lam_s, spatial_eigenvalue_sums(c));
  if (rc) return fail(rc);
  const size_t BN = static_cast<size_t>(c->B) * c->N, BNs = static_cast<size_t>(c->B) * c->Ns;
  double **vecs[] = {&c->r, &c->p, &c->q, &c->z, &c->fd_tmp[0], &c->fd_tmp[1], &c->dF, &c->du};
  for (double **v : vecs)
    if (!rc) rc = dev_alloc(c, v, BN);
  for (int a = 0; a < 8 && !rc; ++a) rc = dev_alloc(c, &c->a64.abuf[a], BN);
  if (!rc) rc = dev_alloc(c, &c->a64.ls_buf, BNs);
  if (df) {  // the double-float A x shares the FP64 A x buffers (same element size)
    for (int a = 0; a < 8; ++a) c->adf.abuf[a] = reinterpret_cast<stls::dfloat *>(c->a64.abuf[a]);
    c->adf.ls_buf = reinterpret_cast<stls::dfloat *>(c->a64.ls_buf);
  }
  if (refine) {
    // the direction-1/2 states of the FP32 product may be stored with every
    // (t, i_3) slice padded to a multiple of 4 values
    size_t BN32 = BN;
    if (c->d == 3)
      BN32 = std::max(BN, static_cast<size_t>(c->B) * c->n_t * c->n_s[2] *
                              ((static_cast<size_t>(c->n_s[0]) * c->n_s[1] + 3) / 4 * 4));
    for (int a = 0; a < 8 && !rc; ++a) rc = dev_alloc(c, &c->a32.abuf[a], BN32);
    if (!rc) rc = dev_alloc(c, &c->a32.ls_buf, BNs);
    float **iv[] = {&c->ri, &c->pi, &c->qi, &c->zi, &c->di};
    for (float **v : iv)
      if (!rc) rc = dev_alloc(c, v, BN);
    if (!rc) rc = dev_alloc(c, &c->st_in, c->B);
    if (!rc) rc = dev_alloc(c, &c->alpha_partials, static_cast<size_t>(c->B) * stls::alpha_blocks(c->Ns));
    if (!rc) rc = dev_alloc(c, &c->alpha_tickets, c->B);
  }
  for (int a = 0; a < 4 && !rc; ++a) rc = dev_alloc(c, &c->lift_tmp[a], BNs);
  if (!rc && geo && P.geo_precond == 0) {
    // D = diag(A) / diag(Pbar^G) from the 1D diagonals; the apply scales by D^{-1/2}
    rc = dev_alloc(c, &c->geo_tmp, BN);
    if (!rc) rc = upload(c, &c->geo_dinv, geometry_scaling(c));
  }
  if (!rc) rc = dev_alloc(c, &c->st, c->B);
  if (!rc) rc = dev_alloc(c, &c->vec_ab, 2 * static_cast<size_t>(c->B));
  if (!rc) rc = dev_alloc(c, &c->vec_out, c->B);
  c->rw.grid = stls::red_grid_for(c->N);
  if (!rc) rc = dev_alloc(c, &c->rw.partials, static_cast<size_t>(c->B) * c->rw.grid * 2);
  if (!rc) rc = dev_alloc(c, &c->rw.tickets, c->B);
  if (rc) return fail(rc);
  if (cudaMallocHost(&c->st_host, sizeof(CGState) * c->B) != cudaSuccess) {
    c->st_host = nullptr;
    c->err = "cudaMallocHost failed";
    return fail(STLS_ENOMEM);
  }
  if (cudaMemset(c->rw.tickets, 0, sizeof(unsigned) * c->B) != cudaSuccess ||
      cudaMemset(c->st, 0, sizeof(CGState) * c->B) != cudaSuccess ||
      (c->st_in != nullptr && cudaMemset(c->st_in, 0, sizeof(CGState) * c->B) != cudaSuccess) ||
      (c->alpha_tickets != nullptr && cudaMemset(c->alpha_tickets, 0, sizeof(unsigned) * c->B) != cudaSuccess)) {
    c->err = "cudaMemset failed";
    return fail(STLS_ECUDA);
  }
  if (P.precision != STLS_FP64) {
    std::vector<std::vector<double>> U(c->d + 1), lam(c->d + 1);
    std::vector<int> n(c->d + 1);
    for (int k = 0; k < c->d; ++k) {
      U[k] = c->hs.eig_s[k].U;
      lam[k] = c->hs.eig_s[k].lam;
      n[k] = c->n_s[k];
    }
    U[c->d] = c->hs.eig_t.U;
    lam[c->d] = c->hs.eig_t.lam;
    n[c->d] = c->n_t;
    std::string tcerr;
    cudaError_t e = stls::tc_fd_create(c->tc, P.precision, c->d, n.data(), c->B, U, lam, c->lam_t, c->lam_s,
                                       tcerr);
    if (e != cudaSuccess || !tcerr.empty()) {
      c->err = tcerr.empty() ? std::string("tensor-core FD setup: ") + cudaGetErrorString(e) : tcerr;
      return fail(tcerr.empty() ? STLS_ECUDA : STLS_EINVAL);
    }
  }
  if (cudaDeviceSynchronize() != cudaSuccess) {
    c->err = "device synchronize after setup failed";
    return fail(STLS_ECUDA);
  }
  *out = c;
  return STLS_OK;
}

int stls_set_stream(stls_ctx *c, void *cuda_stream) {
  if (c == nullptr) return STLS_EINVAL;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  return STLS_OK;
}

int stls_sizes(const stls_ctx *c, int *n_s, int *n_t, long long *n_dof, int *batch) {
  if (c == nullptr) return STLS_EINVAL;
  if (n_s)
    for (int k = 0; k < c->d; ++k) n_s[k] = c->n_s[k];
  if (n_t) *n_t = c->n_t;
  if (n_dof) *n_dof = c->N;
  if (batch) *batch = c->B;
  return STLS_OK;
}

int stls_apply_A(stls_ctx *c, const double *x, double *y) {
  if (c == nullptr) return STLS_EINVAL;
  if (check_ptr(c, x, "x") || check_ptr(c, y, "y")) return STLS_EINVAL;
  if (x == y) return set_err(c, STLS_EINVAL, "apply_A: x and y must not overlap");
  return apply_A_impl<double>(c, c->a64, x, y);
}

int stls_apply_A_df(stls_ctx *c, const double *x, double *y) {
  if (c == nullptr) return STLS_EINVAL;
  if (check_ptr(c, x, "x") || check_ptr(c, y, "y")) return STLS_EINVAL;
  if (x == y) return set_err(c, STLS_EINVAL, "apply_A_df: x and y must not overlap");
  if (!c->have_df) return set_err(c, STLS_EINVAL, "apply_A_df needs a refinement context with d = 2 or 3");
  stls::dfloat *xd = reinterpret_cast<stls::dfloat *>(c->p), *yd = reinterpret_cast<stls::dfloat *>(c->z);
  STLS_LAUNCH(stls::launch_df_split(x, xd, c->N, c->B, nullptr, c->stream), "df_split");
  int rc = apply_A_df_impl(c, xd, yd);
  if (rc) return rc;
  STLS_LAUNCH(stls::launch_df_join(yd, y, c->N, c->B, nullptr, c->stream), "df_join");
  return STLS_OK;
}

int stls_apply_A_f32(stls_ctx *c, const float *x, float *y) {
  if (c == nullptr) return STLS_EINVAL;
  if (x == nullptr || y == nullptr || (reinterpret_cast<uintptr_t>(x) & 3u) != 0 ||
      (reinterpret_cast<uintptr_t>(y) & 3u) != 0)
    return set_err(c, STLS_EINVAL, "apply_A_f32: x or y is NULL or not 4-byte aligned");
  if (x == y) return set_err(c, STLS_EINVAL, "apply_A_f32: x and y must not overlap");
  if (!c->hs.prm.refine || c->a32.abuf[0] == nullptr)
    return set_err(c, STLS_EINVAL, "apply_A_f32 needs a refinement context");
  return apply_A_impl<float>(c, c->a32, x, y);
}

int stls_apply_precond(stls_ctx *c, const double *r, double *z) {
  if (c == nullptr) return STLS_EINVAL;
  if (check_ptr(c, r, "r") || check_ptr(c, z, "z")) return STLS_EINVAL;
  return fd_apply_impl(c, r, z);
}

int stls_solve(stls_ctx *c, const double *F, double *u, double tol, int maxit, stls_solve_info *info) {
  NvtxScope range("stls_solve");
  if (c == nullptr) return STLS_EINVAL;
  if (F == u) return set_err(c, STLS_EINVAL, "solve: F and u must not overlap");
  return c->hs.prm.refine ? solve_ir_impl(c, F, u, tol, maxit, info) : solve_impl(c, F, u, tol, maxit, info);
}

int stls_solve_host(stls_ctx *c, const double *F_host, double *u_host, double tol, int maxit,
                    stls_solve_info *info) {
  NvtxScope range("stls_solve_host");
  if (c == nullptr || F_host == nullptr || u_host == nullptr) return set_err(c, STLS_EINVAL, "NULL argument");
  const size_t bytes = sizeof(double) * static_cast<size_t>(c->B) * c->N;
  if (c->hs.prm.refine && c->copy_stream == nullptr) {
    STLS_CK(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking), "copy stream");
    STLS_CK(cudaEventCreateWithFlags(&c->ev_u, cudaEventDisableTiming), "event");
    STLS_CK(cudaEventCreateWithFlags(&c->ev_copied, cudaEventDisableTiming), "event");
  }
  c->early_issued = c->early_final = false;
  STLS_CK(cudaMemcpyAsync(c->dF, F_host, bytes, cudaMemcpyHostToDevice, c->stream), "H2D copy of F");
  int rc = c->hs.prm.refine ? solve_ir_impl(c, c->dF, c->du, tol, maxit, info, u_host)
                            : solve_impl(c, c->dF, c->du, tol, maxit, info);
  // an early copy of u (refinement form) ends before anything else writes u_host
  if (c->early_issued) STLS_CK(cudaStreamWaitEvent(c->stream, c->ev_copied, 0), "event wait");
  if (rc != STLS_OK && rc != STLS_ENOTCONV && rc != STLS_EBREAKDOWN && rc != STLS_ENONFINITE) {
    cudaStreamSynchronize(c->stream);
    return rc;
  }
  if (!c->early_final)
    STLS_CK(cudaMemcpyAsync(u_host, c->du, bytes, cudaMemcpyDeviceToHost, c->stream), "D2H copy of u");
  STLS_CK(cudaStreamSynchronize(c->stream), "sync");
  return rc;
}

int stls_round_bf16(const double *x, double *y, long long n, void *cuda_stream) {
  if (n < 0 || (n > 0 && (x == nullptr || y == nullptr))) {
    g_create_error = "stls_round_bf16: n < 0 or NULL pointer";
    return STLS_EINVAL;
  }
  cudaError_t e = stls::round_bf16_launch(x, y, n, static_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess) {
    g_create_error = std::string("stls_round_bf16: ") + cudaGetErrorString(e);
    return STLS_ECUDA;
  }
  return STLS_OK;
}

int stls_apply_lift(stls_ctx *c, const double *c0, double *y) {
  if (c == nullptr) return STLS_EINVAL;
  if (is_geometry(c)) return set_err(c, STLS_EINVAL, "lifting calls need geometry = 0");
  if (check_ptr(c, c0, "c0") || check_ptr(c, y, "y")) return STLS_EINVAL;
  double *Js = c->lift_tmp[0], *Ls = c->lift_tmp[1];
  int rc = spatial_tree<double>(c, c->a64, c0, c->B, nullptr, Js, Ls, nullptr);
  if (rc) return rc;
  STLS_LAUNCH(stls::launch_lift_combine(Ls, Js, c->e_end, c->m_int, y, c->Ns, c->n_t, c->B, c->stream),
              "lift_combine");
  return STLS_OK;
}

int stls_lifted_rhs(stls_ctx *c, const double *F, const double *c0, double *rhs) {
  if (c == nullptr) return STLS_EINVAL;
  if (is_geometry(c)) return set_err(c, STLS_EINVAL, "lifting calls need geometry = 0");
  if (check_ptr(c, F, "F") || check_ptr(c, c0, "c0") || check_ptr(c, rhs, "rhs")) return STLS_EINVAL;
  if (rhs == F || rhs == c0) return set_err(c, STLS_EINVAL, "lifted_rhs: rhs must not overlap F or c0");
  double *Gc0 = c->fd_tmp[0];  // B x N workspace
  int rc = stls_apply_lift(c, c0, Gc0);
  if (rc) return rc;
  STLS_LAUNCH(stls::launch_axpy(F, Gc0, -1.0, rhs, static_cast<long long>(c->B) * c->N, c->stream), "axpy");
  return STLS_OK;
}

int stls_lift_add(stls_ctx *c, const double *w, const double *c0, double *u) {
  if (c == nullptr) return STLS_EINVAL;
  if (is_geometry(c)) return set_err(c, STLS_EINVAL, "lifting calls need geometry = 0");
  if (check_ptr(c, w, "w") || check_ptr(c, c0, "c0") || check_ptr(c, u, "u")) return STLS_EINVAL;
  if (u == w || u == c0) return set_err(c, STLS_EINVAL, "lift_add: u must not overlap w or c0");
  // 1_{n_t} x c0 (+ 0 x c0) into the B x N workspace, then u = w + it
  double *y = c->fd_tmp[0];
  STLS_LAUNCH(stls::launch_lift_combine(c0, c0, c->ones_t, c->zeros_t, y, c->Ns, c->n_t, c->B, c->stream),
              "lift_combine");
  STLS_LAUNCH(stls::launch_axpy(w, y, 1.0, u, static_cast<long long>(c->B) * c->N, c->stream), "axpy");
  return STLS_OK;
}

int stls_lift_adjoint(stls_ctx *c, const double *g, const double *lam, double *dc0) {
  if (c == nullptr) return STLS_EINVAL;
  if (is_geometry(c)) return set_err(c, STLS_EINVAL, "lifting calls need geometry = 0");
  if (check_ptr(c, g, "g") || check_ptr(c, lam, "lam") || check_ptr(c, dc0, "dc0")) return STLS_EINVAL;
  // G^T lam = L_s (sum_t e_t lam_t) + J_s (sum_t m_t lam_t)   (L_s, J_s symmetric)
  double *a = c->lift_tmp[0], *bs = c->lift_tmp[1], *gs = c->lift_tmp[2];
  STLS_LAUNCH(stls::launch_lift_reduce(lam, g, c->e_end, c->m_int, a, bs, gs, c->Ns, c->n_t, c->B,
                                       c->stream),
              "lift_reduce");
  double *La = c->a64.ls_buf;       // B x N_s
  double *Jb = c->lift_tmp[3];
  int rc = spatial_tree<double>(c, c->a64, a, c->B, nullptr, nullptr, La, nullptr);
  if (rc) return rc;
  rc = spatial_tree<double>(c, c->a64, bs, c->B, nullptr, Jb, nullptr, nullptr);
  if (rc) return rc;
  const long long n = static_cast<long long>(c->B) * c->Ns;
  STLS_LAUNCH(stls::launch_axpy(gs, La, -1.0, dc0, n, c->stream), "axpy");
  STLS_LAUNCH(stls::launch_axpy(dc0, Jb, -1.0, dc0, n, c->stream), "axpy");
  return STLS_OK;
}

// ---- local operations of a time-slab decomposition -------------------------------------
static int slab_check(stls_ctx *c, const char *what) {
  if (c->hs.prm.precision != STLS_FP64 || is_geometry(c))
    return set_err(c, STLS_EINVAL, std::string(what) + ": FP64 contexts with geometry = 0 only");
  return STLS_OK;
}

int stls_slab_spatial(stls_ctx *c, const double *x, long long ns, double *Ms, double *Js, double *Ls) {
  if (c == nullptr) return STLS_EINVAL;
  if (int rc = slab_check(c, "slab_spatial")) return rc;
  if (check_ptr(c, x, "x")) return STLS_EINVAL;
  if (ns < 1 || ns > static_cast<long long>(c->B) * c->n_t)
    return set_err(c, STLS_EINVAL, "slab_spatial: ns must be in [1, B n_t]");
  if (Ms == nullptr && Js == nullptr && Ls == nullptr) return STLS_OK;
  return spatial_tree<double>(c, c->a64, x, ns, Ms, Js, Ls, nullptr);
}

int stls_slab_time(stls_ctx *c, const double *Ms_ext, const double *Js_ext, int e0, int e1, int t0, int t1,
                   const double *Ls_last, double *y) {
  if (c == nullptr) return STLS_EINVAL;
  if (int rc = slab_check(c, "slab_time")) return rc;
  if (check_ptr(c, Ms_ext, "Ms_ext") || check_ptr(c, Js_ext, "Js_ext") || check_ptr(c, y, "y")) return STLS_EINVAL;
  const int pt = c->hs.prm.p_t, nt = c->n_t;
  if (!(0 <= e0 && e0 <= t0 && t0 < t1 && t1 <= e1 && e1 <= nt) || e0 > std::max(0, t0 - pt) ||
      e1 < std::min(nt, t1 + pt))
    return set_err(c, STLS_EINVAL, "slab_time: need 0 <= e0 <= t0 < t1 <= e1 <= n_t and halos of p_t slices");
  if (t1 == nt && check_ptr(c, Ls_last, "Ls_last")) return STLS_EINVAL;
  const int ne = e1 - e0, w = 2 * pt + 1;
  // the time band on the extended rows (global rows e0 .. e1-1); rows whose band
  // reaches past the extension are wrong and not kept
  double *work = c->fd_tmp[0];
  stls::BandSpec s{};
  s.p = pt;
  s.in[0] = Ms_ext;
  s.in[1] = Js_ext;
  s.n_in = 2;
  s.out[0] = work;
  s.n_out = 1;
  s.term[0] = {c->a64.band_Kt + static_cast<size_t>(e0) * w, 0, 0, 1.0};
  s.term[1] = {c->a64.band_Mt + static_cast<size_t>(e0) * w, 1, 0, 1.0};
  s.n_terms = 2;
  if (t1 == nt) {  // W_t x L_s on the last time slice (the last extended row)
    s.last_add = Ls_last;
    s.last_out = 0;
  }
  ModeView v{};
  v.n = ne;
  v.inner = c->Ns;
  v.outer = c->B;
  v.in_outer_stride = v.out_outer_stride = static_cast<long long>(ne) * c->Ns;
  STLS_LAUNCH(stls::launch_banded(s, v, c->stream), "banded(time slab)");
  const size_t row = sizeof(double) * static_cast<size_t>(c->Ns);
  STLS_CK(cudaMemcpy2DAsync(y, row * (t1 - t0), work + static_cast<size_t>(t0 - e0) * c->Ns, row * ne,
                            row * (t1 - t0), c->B, cudaMemcpyDeviceToDevice, c->stream),
          "slab_time copy");
  return STLS_OK;
}

int stls_fd_spatial(stls_ctx *c, const double *x, double *y, long long ns, int forward) {
  if (c == nullptr) return STLS_EINVAL;
  if (int rc = slab_check(c, "fd_spatial")) return rc;
  if (check_ptr(c, x, "x") || check_ptr(c, y, "y")) return STLS_EINVAL;
  if (x == y) return set_err(c, STLS_EINVAL, "fd_spatial: x and y must not overlap");
  if (ns < 1 || ns > static_cast<long long>(c->B) * c->n_t)
    return set_err(c, STLS_EINVAL, "fd_spatial: ns must be in [1, B n_t]");
  const double *src = x;
  for (int k = 0; k < c->d; ++k) {
    double *dst = k == c->d - 1 ? y : c->fd_tmp[k % 2];
    STLS_LAUNCH(stls::launch_modeprod_f64(src, dst, forward ? c->Uf[k] : c->Ub[k], spatial_view(c, k, ns),
                                          nullptr, nullptr, c->stream),
                "modeprod (spatial)");
    src = dst;
  }
  return STLS_OK;
}

int stls_fd_time_chunk(stls_ctx *c, const double *x, double *y, long long s0, long long s1) {
  if (c == nullptr) return STLS_EINVAL;
  if (int rc = slab_check(c, "fd_time_chunk")) return rc;
  if (check_ptr(c, x, "x") || check_ptr(c, y, "y")) return STLS_EINVAL;
  if (x == y) return set_err(c, STLS_EINVAL, "fd_time_chunk: x and y must not overlap");
  if (!(0 <= s0 && s0 < s1 && s1 <= c->Ns)) return set_err(c, STLS_EINVAL, "fd_time_chunk: need 0 <= s0 < s1 <= N_s");
  ModeView v{};
  v.n = c->n_t;
  v.inner = s1 - s0;
  v.outer = c->B;
  v.in_outer_stride = v.out_outer_stride = static_cast<long long>(c->n_t) * (s1 - s0);
  const int d = c->d;
  STLS_LAUNCH(stls::launch_modeprod_f64(x, c->fd_tmp[0], c->Uf[d], v, c->lam_t, c->lam_s + s0, c->stream),
              "modeprod (time, divide)");
  STLS_LAUNCH(stls::launch_modeprod_f64(c->fd_tmp[0], y, c->Ub[d], v, nullptr, nullptr, c->stream),
              "modeprod (time)");
  return STLS_OK;
}

int stls_vec_dot(stls_ctx *c, const double *x, const double *y, long long n, double *out_host) {
  if (c == nullptr) return STLS_EINVAL;
  if (check_ptr(c, x, "x") || check_ptr(c, y, "y") || out_host == nullptr || n < 0)
    return set_err(c, STLS_EINVAL, "vec_dot: NULL or misaligned pointer, or n < 0");
  STLS_LAUNCH(stls::launch_vec_dot(x, y, n, c->B, c->vec_out, c->rw, c->stream), "vec_dot");
  STLS_CK(cudaMemcpyAsync(out_host, c->vec_out, sizeof(double) * c->B, cudaMemcpyDeviceToHost, c->stream),
          "vec_dot copy");
  STLS_CK(cudaStreamSynchronize(c->stream), "sync");
  return STLS_OK;
}

int stls_vec_axpby(stls_ctx *c, const double *a_host, const double *x, const double *b_host, double *y,
                   long long n) {
  if (c == nullptr) return STLS_EINVAL;
  if (check_ptr(c, x, "x") || check_ptr(c, y, "y") || a_host == nullptr || b_host == nullptr || n < 0)
    return set_err(c, STLS_EINVAL, "vec_axpby: NULL or misaligned pointer, or n < 0");
  const size_t bytes = sizeof(double) * c->B;
  STLS_CK(cudaMemcpyAsync(c->vec_ab, a_host, bytes, cudaMemcpyHostToDevice, c->stream), "vec_axpby upload");
  STLS_CK(cudaMemcpyAsync(c->vec_ab + c->B, b_host, bytes, cudaMemcpyHostToDevice, c->stream), "vec_axpby upload");
  STLS_LAUNCH(stls::launch_vec_axpby(c->vec_ab, x, y, n, c->B, c->stream), "vec_axpby");
  return STLS_OK;
}

int stls_override_eigenvalues(stls_ctx *c, int dir, const double *lam_host) {
  if (c == nullptr) return STLS_EINVAL;
  if (c->hs.prm.precision != STLS_FP64)
    return set_err(c, STLS_EINVAL, "override_eigenvalues: FP64 contexts only");
  if (dir < 0 || dir > c->d || lam_host == nullptr)
    return set_err(c, STLS_EINVAL, "override_eigenvalues: dir out of range or NULL values");
  // work already queued may still read the eigenvalues
  STLS_CK(cudaStreamSynchronize(c->stream), "sync");
  if (dir == c->d) {
    std::vector<double> &lam = c->hs.eig_t.lam;
    std::copy(lam_host, lam_host + lam.size(), lam.begin());
    STLS_CK(cudaMemcpy(c->lam_t, lam.data(), lam.size() * sizeof(double), cudaMemcpyHostToDevice), "upload");
  } else {
    std::vector<double> &lam = c->hs.eig_s[dir].lam;
    std::copy(lam_host, lam_host + lam.size(), lam.begin());
    const std::vector<double> ls = spatial_eigenvalue_sums(c);
    STLS_CK(cudaMemcpy(c->lam_s, ls.data(), ls.size() * sizeof(double), cudaMemcpyHostToDevice), "upload");
  }
  return STLS_OK;
}

int stls_residual_history(const stls_ctx *c, int b, double *host_out, int max_len, int *len) {
  if (c == nullptr || b < 0 || b >= c->B || len == nullptr || max_len < 0) return STLS_EINVAL;
  static const std::vector<double> kNone;
  const std::vector<double> &h = b < static_cast<int>(c->hist.size()) ? c->hist[b] : kNone;
  *len = static_cast<int>(h.size());
  if (host_out != nullptr) std::copy(h.begin(), h.begin() + std::min<size_t>(h.size(), max_len), host_out);
  return STLS_OK;
}

int stls_get_factor(const stls_ctx *c, int which, int dir, double *host_out) {
  if (c == nullptr) return STLS_EINVAL;
  return stls::copy_factor_public(c->hs, which, dir, host_out);
}

long long stls_launch_count(const stls_ctx *c) { return c == nullptr ? 0 : c->launches; }

int stls_enable_timing(stls_ctx *c, int on) {
  if (c == nullptr) return STLS_EINVAL;
  c->timing = on != 0;
  for (int i = 0; i < 5; ++i) {
    c->phase_ms[i] = 0.0;
    c->phase_count[i] = 0;
  }
  c->ev_pairs.clear();
  return STLS_OK;
}

int stls_phase_times(stls_ctx *c, double *ms_out4, long long *count_out4) {
  return stls_phase_times_n(c, 4, ms_out4, count_out4);
}

int stls_phase_times_n(stls_ctx *c, int n, double *ms_out, long long *count_out) {
  if (c == nullptr || n < 0) return STLS_EINVAL;
  for (int i = 0; i < n && i < 5; ++i) {
    if (ms_out) ms_out[i] = c->phase_ms[i];
    if (count_out) count_out[i] = c->phase_count[i];
  }
  return STLS_OK;
}

}  // extern "C"
