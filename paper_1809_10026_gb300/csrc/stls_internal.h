// Internal declarations shared by the host setup, the kernels and the C ABI.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/stls.h"

namespace stls {

constexpr int kMaxDeg = 10;     // largest supported spline degree
constexpr int kMaxDense = 128;  // largest 1D size of the FD mode-product kernels

// One parametric direction with its reduced 1D matrices (Sec. 2.2, 4.1, 4.2).
struct Dir1D {
  int n_el = 0, p = 0, m = 0, n = 0;  // elements, degree, full and reduced sizes
  bool is_time = false;
  double length = 1.0;                // 1 in space, T in time
  std::vector<double> knots;
  std::vector<double> M, K, J;        // reduced n x n, row-major
  std::vector<double> end_values;     // reduced basis at the right end
  std::vector<double> integrals;      // integrals of the reduced basis
};

// Generalized eigendecomposition J U = M U diag(lam), U^T M U = I, lam ascending.
struct Eig1D {
  int n = 0;
  std::vector<double> U, lam;
};

// Weighted 1D factors of the least-squares matrix on the mapped cube
// (geometry = 1; g = g_k of the stretch map, L b = (1/g') (b' / g')').
struct GeoDir {
  std::vector<double> M, K, J, E;  // int b b g', int b' b' / g', int (Lb)(Lb) g', int (L b_i) b_j g'
};

// Host-side description of a problem: directions, pencils, banded factors.
struct HostSetup {
  stls_params prm{};
  std::vector<Dir1D> space;  // d entries
  Dir1D time;                // physical time matrices on [0, T]
  Dir1D time_pencil;         // time matrices used by P (physical or parametric)
  std::vector<Eig1D> eig_s;  // d entries: pencils of the preconditioner
  Eig1D eig_t;
  std::vector<GeoDir> geo;   // geometry = 1: d entries
  // geometry = 1, geo_precond != 2: the 1D matrices of Pbar^G (Sec. 4.4)
  std::vector<std::vector<double>> pg_M, pg_J;  // d entries
  std::vector<double> pg_Mt, pg_Kt;
};

// Separation of variables (App. A.3) for coefficient tensors in product form:
// C^(k)[i_1..i_D] = prod_l F[k][l][i_l] with positive factors.  Writes the
// univariate factors mu[l], omega[l] (lengths of F[0][l]); maxit sweeps.
void separate_product_form(const std::vector<std::vector<std::vector<double>>> &F, int maxit,
                           std::vector<std::vector<double>> &mu, std::vector<std::vector<double>> &omega);

// Returns "" on success or an error message.
std::string validate_params(const stls_params &prm);
Dir1D build_direction(int n_el, int p, bool is_time, double length);
bool generalized_eig(int n, const double *Jm, const double *Mm, Eig1D &out, std::string &err);
bool build_setup(const stls_params &prm, HostSetup &hs, std::string &err);
// Band storage of a reduced matrix: band[i*(2p+1) + o] = A[i][i+o-p] (0 outside).
std::vector<double> to_band(const std::vector<double> &A, int n, int p);

}  // namespace stls
