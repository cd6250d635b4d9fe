// Tensor-core fast-diagonalization solve (Algorithm 1, steps 2-4) for the
// mixed-precision form: mode products with TF32 or BF16 operands and FP32
// accumulation in tensor memory (tcgen05), FP64 input/output and FP64
// eigenvalue division.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

namespace stls {

struct TcFd {
  int precision = 0, d = 0, B = 0;
  int n[4] = {0, 0, 0, 0};
  long long Ns = 0, N = 0;
  int launches_per_apply = 0;
  std::vector<void *> allocations;
  void *impl = nullptr;
};

// U[k] (row-major n[k] x n[k], k = 0..d-1 space, d = time) are the FP64
// eigenvector matrices; lam_t_dev / lam_s_dev are device arrays of the time
// eigenvalues and the summed spatial eigenvalues (length N_s).
cudaError_t tc_fd_create(TcFd &tc, int precision, int d, const int *n, int B,
                         const std::vector<std::vector<double>> &U, const double *lam_t_dev,
                         const double *lam_s_dev, std::string &err);
cudaError_t tc_fd_apply(TcFd &tc, const double *r, double *z, cudaStream_t s);
// Same with FP32 r and z (inner solves of the refinement form).
cudaError_t tc_fd_apply_f32(TcFd &tc, const float *r, float *z, cudaStream_t s);
int tc_fd_launch_count(const TcFd &tc);
// Non-zero once a tensor-core kernel gave up on a bounded wait (host-mapped
// flag; read it after synchronizing the stream).
int tc_fd_error(const TcFd &tc);
void tc_fd_destroy(TcFd &tc);

}  // namespace stls
