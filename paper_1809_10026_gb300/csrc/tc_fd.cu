// Placeholder for the tensor-core FD path; filled in by the tcgen05 kernels.
#include "tc_fd.h"

namespace stls {

cudaError_t tc_fd_create(TcFd &tc, int precision, int d, const int *n, int B,
                         const std::vector<std::vector<double>> &U, const double *lam_t_dev,
                         const double *lam_s_dev, std::string &err) {
  (void)tc; (void)precision; (void)d; (void)n; (void)B; (void)U; (void)lam_t_dev; (void)lam_s_dev;
  err = "mixed precision is not available in this build";
  return cudaSuccess;
}
cudaError_t tc_fd_apply(TcFd &, const double *, double *, cudaStream_t) { return cudaErrorNotSupported; }
int tc_fd_launch_count(const TcFd &tc) { return tc.launches_per_apply; }
void tc_fd_destroy(TcFd &tc) {
  for (void *p : tc.allocations) cudaFree(p);
  tc.allocations.clear();
}

}  // namespace stls
