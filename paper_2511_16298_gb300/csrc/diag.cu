// Failure-detection check of the cross-block waits (tdgs_diag_barrier_timeout):
// of two blocks only block 1 reaches the radix passes' grid barrier, so its
// bounded wait runs out and latches TDGS_ERR_TIMEOUT -- no fault, no hang.
#include "radix.cuh"

namespace tdgs {

namespace {
__global__ void k_diag_barrier_timeout(uint32_t* bar, uint32_t* err) {
  if (blockIdx.x == 1) radix::grid_barrier(bar, err);
}
}  // namespace

cudaError_t launch_diag_barrier_timeout(uint32_t* bar, uint32_t* err, cudaStream_t s) {
  k_diag_barrier_timeout<<<2, 32, 0, s>>>(bar, err);
  return cudaGetLastError();
}

}  // namespace tdgs
