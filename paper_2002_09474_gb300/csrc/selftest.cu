// Self-test of the device-side failure detection: a bounded wait on an
// mbarrier phase that nothing completes.  The wait gives up after its limit
// (kWaitLimitNs of %globaltimer), the kernel records kDevErrTmaTimeout in
// the device error word that morph_device_error() reports, and returns: the
// same path a kernel takes when a TMA load never lands, made without any
// fault, trap or unbounded spin.
#include "morph_common.cuh"
#include "morph_internal.h"

namespace morph {

namespace {

__global__ void __launch_bounds__(32) wait_timeout_kernel(int* err) {
  __shared__ __align__(8) uint64_t bar;
  const int lane = threadIdx.x & 31;
  if (lane == 0) {
    mbar_init(&bar, 1);  // count 1, and no thread ever arrives
    fence_barrier_init();
  }
  __syncwarp();
  const bool landed = mbar_wait_bounded(&bar, 0);
  if (!__any_sync(0xffffffffu, landed) && lane == 0) atomicExch(err, kDevErrTmaTimeout);
}

}  // namespace

cudaError_t selftest_wait_timeout(cudaStream_t stream) {
  int* err = device_error_word();
  if (!err) return cudaErrorInvalidDevice;
  return launch_pdl(false, wait_timeout_kernel, dim3(1), dim3(32), 0, stream, err);
}

}  // namespace morph
