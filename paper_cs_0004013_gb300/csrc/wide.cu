// 64-bit keys as two 32-bit word planes.
//
// A 64-bit key is sorted by eight 8-bit digits, least significant first
// (the LSD scheme of Sec. 3.3.1 with twice the passes).  The passes are the
// key+payload passes of the 32-bit sort: for the four low digits the low
// word is the key and the high word rides along as its payload, for the four
// high digits the roles swap.  Both words of a key always move together, so
// one routing of the eight passes (skipped digits included) keeps the planes
// consistent.  These kernels split the interleaved input into the planes
// (applying the order map of the key kind) and join the planes of the final
// order back into interleaved keys (undoing it).  They serve the persistent
// pass kernels; the tiled ones read and write the interleaved words
// themselves in their first and last executed pass.
#include <cuda_runtime.h>

#include "rs_device.cuh"
#include "rs_internal.h"

namespace rs {

namespace {

__global__ void __launch_bounds__(256) split_kernel(const WideArgs a) {
  const size_t stride = size_t(gridDim.x) * blockDim.x;
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < a.n; i += stride) {
    const uint2 k = map64(a.keys[i], a.x);
    a.lo[i] = k.x;
    a.hi[i] = k.y;
  }
}

__global__ void __launch_bounds__(256) join_kernel(const WideArgs a) {
  const size_t stride = size_t(gridDim.x) * blockDim.x;
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < a.n; i += stride)
    a.out[i] = unmap64(make_uint2(a.lo[i], a.hi[i]), a.x);
}

}  // namespace

cudaError_t launch_split64(const WideArgs& a, unsigned grid, cudaStream_t s) {
  split_kernel<<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_join64(const WideArgs& a, unsigned grid, cudaStream_t s) {
  join_kernel<<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace rs
