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

// Host-side description of a problem: directions, pencils, banded factors.
struct HostSetup {
  stls_params prm{};
  std::vector<Dir1D> space;  // d entries
  Dir1D time;                // physical time matrices on [0, T]
  Dir1D time_pencil;         // time matrices used by P (physical or parametric)
  std::vector<Eig1D> eig_s;  // d entries
  Eig1D eig_t;
};

// Returns "" on success or an error message.
std::string validate_params(const stls_params &prm);
Dir1D build_direction(int n_el, int p, bool is_time, double length);
bool generalized_eig(int n, const double *Jm, const double *Mm, Eig1D &out, std::string &err);
bool build_setup(const stls_params &prm, HostSetup &hs, std::string &err);
// Band storage of a reduced matrix: band[i*(2p+1) + o] = A[i][i+o-p] (0 outside).
std::vector<double> to_band(const std::vector<double> &A, int n, int p);

}  // namespace stls
