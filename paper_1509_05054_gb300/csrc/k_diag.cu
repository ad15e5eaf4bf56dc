// Failure-path diagnostic of the bounded waits.  Every mbarrier wait of the
// tensor-core kernels gives up after a fixed span of the GPU's global timer,
// flags ERR_TIMEOUT in the device error word and lets the kernel return, so a
// lost arrival ends as an error status instead of a hang.  This kernel runs
// exactly that path on purpose: one thread waits on phase 0 of an mbarrier that
// nothing arrives at.
#include "dl_internal.cuh"
#include "tc_ptx.cuh"

namespace dlk {
namespace {

__global__ void wait_timeout_kernel(int* err) {
  __shared__ __align__(8) uint64_t bar;
  tc::mbar_init(&bar, 1);
  if (!tc::mbar_wait(&bar, 0)) atomicOr(err, ERR_TIMEOUT);
}

}  // namespace

cudaError_t bounded_wait_check(int* err, cudaStream_t st) {
  wait_timeout_kernel<<<1, 1, 0, st>>>(err);
  return cudaGetLastError();
}

}  // namespace dlk
