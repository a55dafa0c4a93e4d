// Self-test of the bounded device-side wait: the pass kernels' lookback,
// run on a status row that no tile ever publishes, must give up after its
// round limit, raise the device error word and return (the context stays
// usable; nothing faults or hangs).
#include <cuda_runtime.h>

#include "onesweep.cuh"
#include "rs_internal.h"

namespace rs {
namespace {

__global__ void __launch_bounds__(256) lookback_timeout_kernel(const uint32_t* status, uint32_t* err) {
  uint32_t prefix[1];
  // tile 1 of a segment starting at tile 0: row 0 holds zeroes, which never
  // look ready for parity 1
  lookback<256, 1, uint32_t, 8>(status, 1u, 0u, int(threadIdx.x), 1u, err, prefix);
}

}  // namespace

cudaError_t launch_lookback_timeout(const uint32_t* status, uint32_t* err, cudaStream_t s) {
  lookback_timeout_kernel<<<1, 256, 0, s>>>(status, err);
  return cudaGetLastError();
}

}  // namespace rs
