// Host setup of the solver, FP64 (the "setup" of Sec. 4.5):
//  * uniform open knot vectors (Sec. 2.1),
//  * element-wise Gauss-Legendre quadrature (nodes by Newton's method on the
//    Legendre three-term recurrence),
//  * B-spline values and first/second derivatives by the Cox-de Boor
//    recursion with 0/0 = 0 (Sec. 2.1) and de Boor's derivative formula,
//  * reduced 1D Galerkin matrices M = int b b, K = int b' b', J = int b'' b''
//    (Sec. 4.1, 4.2; space drops the first and last function, time drops
//    the first, Sec. 2.2),
//  * the generalized eigendecompositions of Algorithm 1, step 1, by Cholesky
//    reduction and the cyclic Jacobi method (Golub & Van Loan, Matrix
//    Computations, Sec. 8.5 and 8.7),
//  * for the stretched parametrization of the cube (geometry = 1): the
//    weighted 1D factors of the least-squares matrix on the mapped splines,
//    and the geometry-aware preconditioner of Sec. 4.4 (coefficients at the
//    element barycentres, separation of variables of App. A.3, 1D matrices
//    with element-wise constant weights).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "stls_internal.h"

namespace stls {

std::string validate_params(const stls_params &prm) {
  if (prm.d < 1 || prm.d > 3) return "d must be 1, 2 or 3";
  if (prm.p_s < 2 || prm.p_s > kMaxDeg) return "p_s must be in [2, 10] (C^1 splines in space)";
  if (prm.p_t < 1 || prm.p_t > kMaxDeg) return "p_t must be in [1, 10]";
  if (!(prm.T > 0.0) || !std::isfinite(prm.T)) return "T must be a finite positive number";
  if (prm.n_el_t < 1) return "n_el_t must be >= 1";
  for (int k = 0; k < prm.d; ++k) {
    if (prm.n_el_s[k] < 1) return "n_el_s must be >= 1";
    if (prm.n_el_s[k] + prm.p_s - 2 > kMaxDense) return "spatial size n_el + p - 2 exceeds 128";
  }
  if (prm.n_el_t + prm.p_t - 1 > kMaxDense) return "time size n_el_t + p_t - 1 exceeds 128";
  if (prm.precision < STLS_FP64 || prm.precision > STLS_MIXED_BF16) return "unknown precision";
  if (prm.batch < 1 || prm.batch > 1024) return "batch must be in [1, 1024]";
  if (prm.flexible != 0 && prm.flexible != 1) return "flexible must be 0 or 1";
  if (prm.time_pencil != 0 && prm.time_pencil != 1) return "time_pencil must be 0 or 1";
  if (prm.refine != 0 && prm.refine != 1) return "refine must be 0 or 1";
  if (prm.refine == 1 && prm.precision == STLS_FP64) return "refine = 1 needs a mixed precision form";
  if (!(prm.inner_tol >= 0.0) || !(prm.inner_tol < 1.0)) return "inner_tol must be in [0, 1)";
  if (prm.fp64_residuals != 0 && prm.fp64_residuals != 1) return "fp64_residuals must be 0 or 1";
  if (prm.geometry != 0 && prm.geometry != 1) return "geometry must be 0 or 1";
  if (prm.geometry == 1) {
    if (prm.precision != STLS_FP64) return "geometry = 1 needs precision = STLS_FP64";
    if (prm.geo_precond < 0 || prm.geo_precond > 2) return "geo_precond must be 0, 1 or 2";
    for (int k = 0; k < prm.d; ++k)
      if (!(std::fabs(prm.geo_a[k]) < 1.0)) return "geo_a[k] must satisfy |geo_a[k]| < 1";
  }
  return "";
}

// Gauss-Legendre nodes and weights on [-1, 1].
static void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double pn = 0, dpn = 0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = pk;
      }
      pn = p1;
      dpn = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = pn / dpn;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) {
      double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = pk;
    }
    dpn = n * (z * p1 - p0) / (z * z - 1.0);
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dpn * dpn);
  }
}

// Values (v0) and first (v1) and second (v2) derivatives at x of the p+1
// B-splines of degree p that are non-zero on span s (t[s] <= x <= t[s+1]);
// entry j belongs to global function s - p + j.
static void eval_span(const std::vector<double> &t, int p, int s, double x, double *v0,
                      double *v1, double *v2) {
  double N[kMaxDeg + 1][kMaxDeg + 1];
  std::memset(N, 0, sizeof(N));
  N[0][0] = 1.0;
  for (int q = 1; q <= p; ++q) {
    for (int j = 0; j <= q; ++j) {
      int i = s - q + j;
      double a = 0.0, b = 0.0;
      if (j >= 1) {
        double den = t[i + q] - t[i];
        if (den != 0.0) a = (x - t[i]) / den * N[q - 1][j - 1];
      }
      if (j <= q - 1) {
        double den = t[i + q + 1] - t[i + 1];
        if (den != 0.0) b = (t[i + q + 1] - x) / den * N[q - 1][j];
      }
      N[q][j] = a + b;
    }
  }
  // derivative of the degree-q functions of span s from degree q-1 values `low`
  auto deriv = [&](int q, const double *low, double *out) {
    for (int j = 0; j <= q; ++j) {
      int i = s - q + j;
      double a = 0.0, b = 0.0;
      if (j >= 1) {
        double den = t[i + q] - t[i];
        if (den != 0.0) a = low[j - 1] / den;
      }
      if (j <= q - 1) {
        double den = t[i + q + 1] - t[i + 1];
        if (den != 0.0) b = low[j] / den;
      }
      out[j] = q * (a - b);
    }
  };
  for (int j = 0; j <= p; ++j) v0[j] = N[p][j];
  if (p >= 1) {
    deriv(p, N[p - 1], v1);
  } else {
    v1[0] = 0.0;
  }
  if (p >= 2) {
    double d1low[kMaxDeg + 1];
    deriv(p - 1, N[p - 2], d1low);
    deriv(p, d1low, v2);
  } else {
    for (int j = 0; j <= p; ++j) v2[j] = 0.0;
  }
}

Dir1D build_direction(int n_el, int p, bool is_time, double length) {
  Dir1D D;
  D.n_el = n_el;
  D.p = p;
  D.m = n_el + p;
  D.is_time = is_time;
  D.length = length;
  D.knots.assign(p + 1, 0.0);
  for (int i = 1; i < n_el; ++i) D.knots.push_back(length * i / n_el);
  for (int i = 0; i <= p; ++i) D.knots.push_back(length);
  const int m = D.m;
  std::vector<double> Mf(m * m, 0.0), Kf(m * m, 0.0), Jf(m * m, 0.0), If(m, 0.0);
  std::vector<double> gx, gw;
  gauss_legendre(p + 1, gx, gw);  // exact for every product of two degree-p splines
  double v0[kMaxDeg + 1], v1[kMaxDeg + 1], v2[kMaxDeg + 1];
  for (int s = p; s < m; ++s) {
    double a = D.knots[s], b = D.knots[s + 1];
    if (!(b > a)) continue;
    for (size_t q = 0; q < gx.size(); ++q) {
      double x = 0.5 * (b - a) * gx[q] + 0.5 * (a + b);
      double w = 0.5 * (b - a) * gw[q];
      eval_span(D.knots, p, s, x, v0, v1, v2);
      for (int r = 0; r <= p; ++r) {
        int gi = s - p + r;
        If[gi] += w * v0[r];
        for (int c = 0; c <= p; ++c) {
          int gj = s - p + c;
          Mf[gi * m + gj] += w * v0[r] * v0[c];
          Kf[gi * m + gj] += w * v1[r] * v1[c];
          Jf[gi * m + gj] += w * v2[r] * v2[c];
        }
      }
    }
  }
  // values of the full basis at the right end (left limit on the last span)
  std::vector<double> endf(m, 0.0);
  eval_span(D.knots, p, m - 1, length, v0, v1, v2);
  for (int r = 0; r <= p; ++r) endf[m - 1 - p + r] = v0[r];
  const int first = 1, last = is_time ? m - 1 : m - 2;  // reduced basis, Sec. 2.2
  D.n = last - first + 1;
  const int n = D.n;
  D.M.assign(n * n, 0.0);
  D.K.assign(n * n, 0.0);
  D.J.assign(n * n, 0.0);
  D.end_values.assign(n, 0.0);
  D.integrals.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    D.end_values[i] = endf[first + i];
    D.integrals[i] = If[first + i];
    for (int j = 0; j < n; ++j) {
      D.M[i * n + j] = Mf[(first + i) * m + first + j];
      D.K[i * n + j] = Kf[(first + i) * m + first + j];
      D.J[i * n + j] = Jf[(first + i) * m + first + j];
    }
  }
  return D;
}

// Cholesky factor L (lower, row-major) of the SPD matrix A; false if not SPD.
static bool cholesky(int n, const double *A, std::vector<double> &L) {
  L.assign(n * n, 0.0);
  for (int j = 0; j < n; ++j) {
    double s = A[j * n + j];
    for (int k = 0; k < j; ++k) s -= L[j * n + k] * L[j * n + k];
    if (!(s > 0.0)) return false;
    double ljj = std::sqrt(s);
    L[j * n + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      double v = A[i * n + j];
      for (int k = 0; k < j; ++k) v -= L[i * n + k] * L[j * n + k];
      L[i * n + j] = v / ljj;
    }
  }
  return true;
}

bool generalized_eig(int n, const double *Jm, const double *Mm, Eig1D &out, std::string &err) {
  std::vector<double> L;
  if (!cholesky(n, Mm, L)) {
    err = "mass matrix is not positive definite";
    return false;
  }
  // Y = L^{-1} J (forward substitution, column by column), then C = L^{-1} Y^T.
  std::vector<double> Y(n * n), C(n * n);
  for (int c = 0; c < n; ++c)
    for (int i = 0; i < n; ++i) {
      double v = Jm[i * n + c];
      for (int k = 0; k < i; ++k) v -= L[i * n + k] * Y[k * n + c];
      Y[i * n + c] = v / L[i * n + i];
    }
  for (int c = 0; c < n; ++c)
    for (int i = 0; i < n; ++i) {
      double v = Y[c * n + i];  // (Y^T)[i][c]
      for (int k = 0; k < i; ++k) v -= L[i * n + k] * C[k * n + c];
      C[i * n + c] = v / L[i * n + i];
    }
  for (int i = 0; i < n; ++i)  // symmetrize rounding
    for (int j = i + 1; j < n; ++j) {
      double v = 0.5 * (C[i * n + j] + C[j * n + i]);
      C[i * n + j] = C[j * n + i] = v;
    }
  // Cyclic Jacobi: rotate every off-diagonal entry that is not negligible
  // relative to its diagonal pair, until a sweep makes no rotation.
  std::vector<double> V(n * n, 0.0);
  for (int i = 0; i < n; ++i) V[i * n + i] = 1.0;
  const double eps = 2.220446049250313e-16;
  bool rotated = true;
  int sweeps = 0;
  for (; rotated && sweeps < 60; ++sweeps) {
    rotated = false;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        double apq = C[p * n + q];
        double app = C[p * n + p], aqq = C[q * n + q];
        if (std::fabs(apq) <= eps * std::sqrt(std::fabs(app * aqq)) || apq == 0.0) continue;
        rotated = true;
        double tau = (aqq - app) / (2.0 * apq);
        double tt = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
        double c = 1.0 / std::sqrt(1.0 + tt * tt), s = tt * c;
        for (int k = 0; k < n; ++k) {  // columns p, q of C
          double ckp = C[k * n + p], ckq = C[k * n + q];
          C[k * n + p] = c * ckp - s * ckq;
          C[k * n + q] = s * ckp + c * ckq;
        }
        for (int k = 0; k < n; ++k) {  // rows p, q of C
          double cpk = C[p * n + k], cqk = C[q * n + k];
          C[p * n + k] = c * cpk - s * cqk;
          C[q * n + k] = s * cpk + c * cqk;
        }
        C[p * n + q] = C[q * n + p] = 0.0;
        for (int k = 0; k < n; ++k) {
          double vkp = V[k * n + p], vkq = V[k * n + q];
          V[k * n + p] = c * vkp - s * vkq;
          V[k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  if (rotated) {
    err = "Jacobi eigensolver did not converge";
    return false;
  }
  // U = L^{-T} V (back substitution with L^T), eigenvalues ascending.
  std::vector<double> Uraw(n * n);
  for (int c = 0; c < n; ++c)
    for (int i = n - 1; i >= 0; --i) {
      double v = V[i * n + c];
      for (int k = i + 1; k < n; ++k) v -= L[k * n + i] * Uraw[k * n + c];
      Uraw[i * n + c] = v / L[i * n + i];
    }
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](int a, int b) { return C[a * n + a] < C[b * n + b]; });
  out.n = n;
  out.U.assign(n * n, 0.0);
  out.lam.assign(n, 0.0);
  for (int c = 0; c < n; ++c) {
    out.lam[c] = C[order[c] * n + order[c]];
    for (int i = 0; i < n; ++i) out.U[i * n + c] = Uraw[i * n + order[c]];
  }
  return true;
}

// Derivatives of the stretch map g(s) = s + a sin(2 pi s) / (2 pi).
static double geo_dg(double a, double s) { return 1.0 + a * std::cos(2.0 * M_PI * s); }
static double geo_d2g(double a, double s) { return -2.0 * M_PI * a * std::sin(2.0 * M_PI * s); }

// Weighted factors of one space direction of the mapped cube (reduced basis),
// by 2p + 6 Gauss points per element (the weights are not polynomials).
static GeoDir build_geo_direction(const Dir1D &D, double a) {
  const int p = D.p, m = D.m, n = D.n;
  std::vector<double> Mf(m * m, 0.0), Kf(m * m, 0.0), Jf(m * m, 0.0), Ef(m * m, 0.0);
  std::vector<double> gx, gw;
  gauss_legendre(2 * p + 6, gx, gw);
  double v0[kMaxDeg + 1], v1[kMaxDeg + 1], v2[kMaxDeg + 1], lb[kMaxDeg + 1];
  for (int sp = p; sp < m; ++sp) {
    const double lo = D.knots[sp], hi = D.knots[sp + 1];
    if (!(hi > lo)) continue;
    for (size_t q = 0; q < gx.size(); ++q) {
      const double x = 0.5 * (hi - lo) * gx[q] + 0.5 * (lo + hi);
      const double w = 0.5 * (hi - lo) * gw[q];
      const double g1 = geo_dg(a, x), g2 = geo_d2g(a, x);
      eval_span(D.knots, p, sp, x, v0, v1, v2);
      for (int r = 0; r <= p; ++r) lb[r] = v2[r] / (g1 * g1) - v1[r] * g2 / (g1 * g1 * g1);
      for (int r = 0; r <= p; ++r) {
        const int gi = sp - p + r;
        for (int c = 0; c <= p; ++c) {
          const int gj = sp - p + c;
          Mf[gi * m + gj] += w * g1 * v0[r] * v0[c];
          Kf[gi * m + gj] += w / g1 * v1[r] * v1[c];
          Jf[gi * m + gj] += w * g1 * lb[r] * lb[c];
          Ef[gi * m + gj] += w * g1 * lb[r] * v0[c];
        }
      }
    }
  }
  GeoDir G;
  auto reduce = [&](const std::vector<double> &F, std::vector<double> &out) {
    out.assign(static_cast<size_t>(n) * n, 0.0);
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) out[i * n + j] = F[(1 + i) * m + 1 + j];  // space: drop first and last
  };
  reduce(Mf, G.M);
  reduce(Kf, G.K);
  reduce(Jf, G.J);
  reduce(Ef, G.E);
  return G;
}

// int w_e b^(ord)_i b^(ord)_j with a weight constant on each element e (p+1
// Gauss points per element: exact), on the reduced basis of D.
static std::vector<double> element_weighted(const Dir1D &D, const std::vector<double> &we, int ord) {
  const int p = D.p, m = D.m, n = D.n;
  const int first = 1;
  std::vector<double> Af(m * m, 0.0);
  std::vector<double> gx, gw;
  gauss_legendre(p + 1, gx, gw);
  double v[3][kMaxDeg + 1];
  int e = 0;
  for (int sp = p; sp < m; ++sp) {
    const double lo = D.knots[sp], hi = D.knots[sp + 1];
    if (!(hi > lo)) continue;
    for (size_t q = 0; q < gx.size(); ++q) {
      const double x = 0.5 * (hi - lo) * gx[q] + 0.5 * (lo + hi);
      const double w = 0.5 * (hi - lo) * gw[q] * we[e];
      eval_span(D.knots, p, sp, x, v[0], v[1], v[2]);
      for (int r = 0; r <= p; ++r)
        for (int c = 0; c <= p; ++c) Af[(sp - p + r) * m + sp - p + c] += w * v[ord][r] * v[ord][c];
    }
    ++e;
  }
  std::vector<double> out(static_cast<size_t>(n) * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) out[i * n + j] = Af[(first + i) * m + first + j];
  return out;
}

// App. A.3 in product form.  The omega-update sets omega^(k)_j from the min and
// max over the slice i_k = j of C^(k) / prod_{l != k} mu^(l); the mu-update
// sets mu^(k)_j from the min over the slice of the element-wise minimum, and
// the max of the maximum, over coefficients l != k of C^(l) divided by its
// product approximation and multiplied by mu^(k) (the estimate of mu^(k) that
// c_l gives).  With C^(k) = prod_l F[k][l](i_l), every such min or max over a
// slice is a product of the per-direction minima or maxima.
void separate_product_form(const std::vector<std::vector<std::vector<double>>> &F, int maxit,
                           std::vector<std::vector<double>> &mu, std::vector<std::vector<double>> &omega) {
  const int D = static_cast<int>(F.size());
  mu.assign(D, {});
  omega.assign(D, {});
  for (int l = 0; l < D; ++l) {
    mu[l].assign(F[0][l].size(), 1.0);
    omega[l].assign(F[0][l].size(), 1.0);
  }
  auto minmax_ratio = [](const std::vector<double> &f, const std::vector<double> &g, double &mn, double &mx) {
    mn = f[0] / g[0];
    mx = mn;
    for (size_t i = 1; i < f.size(); ++i) {
      const double r = f[i] / g[i];
      mn = std::min(mn, r);
      mx = std::max(mx, r);
    }
  };
  for (int it = 0; it < maxit; ++it) {
    for (int k = 0; k < D; ++k) {
      double pmin = 1.0, pmax = 1.0;
      for (int l = 0; l < D; ++l) {
        if (l == k) continue;
        double mn, mx;
        minmax_ratio(F[k][l], mu[l], mn, mx);
        pmin *= mn;
        pmax *= mx;
      }
      for (size_t j = 0; j < omega[k].size(); ++j) omega[k][j] = F[k][k][j] * std::sqrt(pmin * pmax);
    }
    for (int k = 0; k < D; ++k) {
      std::vector<double> ymin(mu[k].size(), 0.0), zmax(mu[k].size(), 0.0);
      bool first = true;
      for (int l = 0; l < D; ++l) {
        if (l == k) continue;
        // C^(l) / approx_l * mu^(k): direction l carries F[l][l] / omega^(l),
        // direction k carries F[l][k], every other m carries F[l][m] / mu^(m)
        double pmin, pmax;
        minmax_ratio(F[l][l], omega[l], pmin, pmax);
        for (int m = 0; m < D; ++m) {
          if (m == k || m == l) continue;
          double mn, mx;
          minmax_ratio(F[l][m], mu[m], mn, mx);
          pmin *= mn;
          pmax *= mx;
        }
        for (size_t j = 0; j < mu[k].size(); ++j) {
          const double lo = F[l][k][j] * pmin, hi = F[l][k][j] * pmax;
          ymin[j] = first ? lo : std::min(ymin[j], lo);
          zmax[j] = first ? hi : std::max(zmax[j], hi);
        }
        first = false;
      }
      for (size_t j = 0; j < mu[k].size(); ++j) mu[k][j] = std::sqrt(ymin[j] * zmax[j]);
    }
  }
}

// The 1D matrices of Pbar^G for the stretch map: coefficients of Eq.
// coefficients-c at the element barycentres, c_k = ||J^-1 e_k||^4 |det J| T
// = T g_k'^-3 prod_{l != k} g_l' and c_{d+1} = prod_l g_l' / T (per-direction
// factors, the time factor constant), separated by two sweeps of App. A.3.
static void build_geo_preconditioner(const stls_params &prm, HostSetup &hs) {
  const int d = prm.d, D = d + 1;
  std::vector<std::vector<double>> gp(d);
  for (int k = 0; k < d; ++k) {
    const int ne = prm.n_el_s[k];
    gp[k].resize(ne);
    for (int e = 0; e < ne; ++e) gp[k][e] = geo_dg(prm.geo_a[k], (e + 0.5) / ne);
  }
  std::vector<std::vector<std::vector<double>>> F(D, std::vector<std::vector<double>>(D));
  for (int k = 0; k < D; ++k)
    for (int l = 0; l < D; ++l) {
      if (l == d) {  // time direction: constant factor
        F[k][l].assign(prm.n_el_t, k < d ? prm.T : 1.0 / prm.T);
        continue;
      }
      F[k][l] = gp[l];
      if (k == l)
        for (double &v : F[k][l]) v = 1.0 / (v * v * v);
    }
  std::vector<std::vector<double>> mu, om;
  separate_product_form(F, 2, mu, om);
  hs.pg_M.assign(d, {});
  hs.pg_J.assign(d, {});
  for (int k = 0; k < d; ++k) {
    hs.pg_M[k] = element_weighted(hs.space[k], mu[k], 0);
    hs.pg_J[k] = element_weighted(hs.space[k], om[k], 2);
  }
  const Dir1D th = build_direction(prm.n_el_t, prm.p_t, true, 1.0);  // parametric time
  // the time direction's reduced basis drops only its first function
  auto time_weighted = [&](const std::vector<double> &we, int ord) {
    const int p = th.p, m = th.m, n = th.n;
    std::vector<double> Af(m * m, 0.0), gx, gw;
    gauss_legendre(p + 1, gx, gw);
    double v[3][kMaxDeg + 1];
    int e = 0;
    for (int sp = p; sp < m; ++sp) {
      const double lo = th.knots[sp], hi = th.knots[sp + 1];
      if (!(hi > lo)) continue;
      for (size_t q = 0; q < gx.size(); ++q) {
        const double x = 0.5 * (hi - lo) * gx[q] + 0.5 * (lo + hi);
        const double w = 0.5 * (hi - lo) * gw[q] * we[e];
        eval_span(th.knots, p, sp, x, v[0], v[1], v[2]);
        for (int r = 0; r <= p; ++r)
          for (int c = 0; c <= p; ++c) Af[(sp - p + r) * m + sp - p + c] += w * v[ord][r] * v[ord][c];
      }
      ++e;
    }
    std::vector<double> out(static_cast<size_t>(n) * n, 0.0);
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) out[i * n + j] = Af[(1 + i) * m + 1 + j];
    return out;
  };
  hs.pg_Mt = time_weighted(mu[d], 0);
  hs.pg_Kt = time_weighted(om[d], 1);
}

bool build_setup(const stls_params &prm, HostSetup &hs, std::string &err) {
  err = validate_params(prm);
  if (!err.empty()) return false;
  hs.prm = prm;
  hs.space.clear();
  hs.eig_s.clear();
  for (int k = 0; k < prm.d; ++k) {
    hs.space.push_back(build_direction(prm.n_el_s[k], prm.p_s, false, 1.0));
    Eig1D e;
    const Dir1D &D = hs.space.back();
    if (!generalized_eig(D.n, D.J.data(), D.M.data(), e, err)) return false;
    hs.eig_s.push_back(e);
  }
  hs.time = build_direction(prm.n_el_t, prm.p_t, true, prm.T);
  hs.time_pencil = prm.time_pencil == 0 ? hs.time : build_direction(prm.n_el_t, prm.p_t, true, 1.0);
  const Dir1D &Tp = hs.time_pencil;
  if (!generalized_eig(Tp.n, Tp.K.data(), Tp.M.data(), hs.eig_t, err)) return false;
  hs.geo.clear();
  if (prm.geometry == 1) {
    for (int k = 0; k < prm.d; ++k) hs.geo.push_back(build_geo_direction(hs.space[k], prm.geo_a[k]));
    if (prm.geo_precond != 2) {
      // the preconditioner's pencils are those of Pbar^G
      build_geo_preconditioner(prm, hs);
      for (int k = 0; k < prm.d; ++k) {
        const int n = hs.space[k].n;
        if (!generalized_eig(n, hs.pg_J[k].data(), hs.pg_M[k].data(), hs.eig_s[k], err)) return false;
      }
      if (!generalized_eig(hs.time.n, hs.pg_Kt.data(), hs.pg_Mt.data(), hs.eig_t, err)) return false;
    }
  }
  return true;
}

std::vector<double> to_band(const std::vector<double> &A, int n, int p) {
  const int w = 2 * p + 1;
  std::vector<double> band(static_cast<size_t>(n) * w, 0.0);
  for (int i = 0; i < n; ++i)
    for (int o = 0; o < w; ++o) {
      int j = i + o - p;
      if (j >= 0 && j < n) band[i * w + o] = A[i * n + j];
    }
  return band;
}

}  // namespace stls

// ---- host-only C entry point --------------------------------------------------------
static int copy_factor(const stls::HostSetup &hs, int which, int dir, double *out) {
  const int d = hs.prm.d;
  if (dir < 0 || dir > d || out == nullptr) return STLS_EINVAL;
  const bool is_time = dir == d;
  const stls::Dir1D &D = is_time ? hs.time : hs.space[dir];
  const stls::Eig1D &E = is_time ? hs.eig_t : hs.eig_s[dir];
  const std::vector<double> *src = nullptr;
  switch (which) {
    case STLS_F_MASS: src = &D.M; break;
    case STLS_F_STIFF: src = &D.K; break;
    case STLS_F_BILAP:
      if (is_time) return STLS_EINVAL;
      src = &D.J;
      break;
    case STLS_F_EIGVEC: src = &E.U; break;
    case STLS_F_EIGVAL: src = &E.lam; break;
    case STLS_F_END:
      if (!is_time) return STLS_EINVAL;
      src = &D.end_values;
      break;
    case STLS_F_INTEGRAL: src = &D.integrals; break;
    case STLS_F_GEO_MASS:
    case STLS_F_GEO_STIFF:
    case STLS_F_GEO_BILAP:
    case STLS_F_GEO_E: {
      if (is_time || hs.prm.geometry != 1) return STLS_EINVAL;
      const stls::GeoDir &G = hs.geo[dir];
      src = which == STLS_F_GEO_MASS ? &G.M : which == STLS_F_GEO_STIFF ? &G.K : which == STLS_F_GEO_BILAP ? &G.J : &G.E;
      break;
    }
    default: return STLS_EINVAL;
  }
  std::memcpy(out, src->data(), src->size() * sizeof(double));
  return STLS_OK;
}

namespace stls {
int copy_factor_public(const HostSetup &hs, int which, int dir, double *out) {
  return copy_factor(hs, which, dir, out);
}
}  // namespace stls

namespace stls {
void set_thread_error(const std::string &msg);
}

extern "C" int stls_host_factor(const stls_params *prm, int which, int dir, double *host_out) {
  stls::set_thread_error("");
  if (prm == nullptr) {
    stls::set_thread_error("stls_host_factor: prm is NULL");
    return STLS_EINVAL;
  }
  stls::HostSetup hs;
  std::string err;
  if (!stls::build_setup(*prm, hs, err)) {
    stls::set_thread_error("stls_host_factor: " + err);
    return STLS_EINVAL;
  }
  const int rc = copy_factor(hs, which, dir, host_out);
  if (rc != STLS_OK) stls::set_thread_error("stls_host_factor: unknown factor id or direction for it");
  return rc;
}
