// Tensor-core fast-diagonalization solve (Algorithm 1, steps 2-4) for the
// mixed-precision form: mode products with TF32 or BF16 operands and FP32
// accumulation in tensor memory (tcgen05), FP64 input/output and FP64
// eigenvalue division.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

namespace stls {

// Raises (never lowers) a kernel's dynamic shared-memory limit.  The limit is
// per kernel and per process, so contexts of different sizes share it: a
// smaller context created later must not lower the limit a larger one needs.
template <typename K>
cudaError_t raise_smem_limit(K *kernel, int bytes) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, reinterpret_cast<const void *>(kernel));
  if (e != cudaSuccess) return e;
  if (fa.maxDynamicSharedSizeBytes >= bytes) return cudaSuccess;
  return cudaFuncSetAttribute(reinterpret_cast<const void *>(kernel), cudaFuncAttributeMaxDynamicSharedMemorySize,
                              bytes);
}

struct FusedFd;
struct RotFd;

struct TcFd {
  int precision = 0, d = 0, B = 0;
  int n[4] = {0, 0, 0, 0};
  long long Ns = 0, N = 0;
  int launches_per_apply = 0;
  std::vector<void *> allocations;
  void *impl = nullptr;
  FusedFd *fused = nullptr;  // BF16, d = 2, 3: fused passes (tc_fd_fused.cu)
  RotFd *rot = nullptr;      // TF32: TMA-fed rotation passes (tc_fd_tf32.cu)
};

// U[k] (row-major n[k] x n[k], k = 0..d-1 space, d = time) are the FP64
// eigenvector matrices and lam[k] their eigenvalues; lam_t_dev / lam_s_dev are
// device arrays of the time eigenvalues and the summed spatial eigenvalues
// (length N_s).  BF16 with d = 2 or 3 and every n[k] <= 128 uses the fused
// passes; other cases one launch per mode product.
cudaError_t tc_fd_create(TcFd &tc, int precision, int d, const int *n, int B,
                         const std::vector<std::vector<double>> &U, const std::vector<std::vector<double>> &lam,
                         const double *lam_t_dev, const double *lam_s_dev, std::string &err);
cudaError_t tc_fd_apply(TcFd &tc, const double *r, double *z, cudaStream_t s);
// Same with FP32 r and z (inner solves of the refinement form).
cudaError_t tc_fd_apply_f32(TcFd &tc, const float *r, float *z, cudaStream_t s);
int tc_fd_launch_count(const TcFd &tc);
// TF32 rotation passes only: the padded input buffer (NULL when the context
// has no such passes), and z = P^{-1} r for an r already written there.
float *tc_fd_padded_input(TcFd &tc, int *n0, int *np0);
cudaError_t tc_fd_apply_f32_padded(TcFd &tc, float *z, cudaStream_t s);
// Non-zero once a tensor-core kernel gave up on a bounded wait (host-mapped
// flag; read it after synchronizing the stream).
int tc_fd_error(const TcFd &tc);
// The same flag as a device pointer (NULL without tensor-core passes), for
// kernels that must stop work after a failed wait.
const int *tc_fd_error_flag(const TcFd &tc);
void tc_fd_destroy(TcFd &tc);

// Fused BF16 passes (slab and streaming kernels), tc_fd_fused.cu.
bool tc_fd_fused_eligible(int precision, int d, const int *n);
cudaError_t tc_fd_fused_create(FusedFd *&out, std::vector<void *> &allocs, int d, const int *n, int B,
                               const std::vector<std::vector<double>> &U, const std::vector<std::vector<double>> &lam,
                               int *err_dev, std::string &err);
template <typename IO>
cudaError_t tc_fd_fused_apply(FusedFd *f, const IO *r, IO *z, cudaStream_t s);
int tc_fd_fused_launches(const FusedFd *f);
void tc_fd_fused_destroy(FusedFd *f);
// TF32 rotation passes (tc_fd_tf32.cu): 2(d+1) mode products with TMA-fed
// K-major operands and a padding pass for r.
bool tc_fd_rot_eligible(int precision, int d, const int *n, int B);
cudaError_t tc_fd_rot_create(RotFd *&out, std::vector<void *> &allocs, int d, const int *n, int B,
                             const std::vector<std::vector<double>> &U, const std::vector<std::vector<double>> &lam,
                             int *err_dev, std::string &err);
template <typename IO>
cudaError_t tc_fd_rot_apply(RotFd *f, const IO *r, IO *z, cudaStream_t s);
int tc_fd_rot_launches(const RotFd *f);
// The buffer the first rotation pass reads (rows of n0 FP32 values, np0 apart,
// rounded to TF32), for producers that write r there directly, and the passes
// alone on it.
float *tc_fd_rot_padded_input(RotFd *f, int *n0, int *np0);
cudaError_t tc_fd_rot_apply_padded(RotFd *f, float *z, cudaStream_t s);
void tc_fd_rot_destroy(RotFd *f);
// y = FP64(BF16(FP32(x))), both roundings to nearest even, as the fused kernels round r.
cudaError_t round_bf16_launch(const double *x, double *y, long long n, cudaStream_t s);

}  // namespace stls
