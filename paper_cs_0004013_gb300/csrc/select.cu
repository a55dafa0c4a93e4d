// The selection step of Sec. 4.2.1: before committing to the bucketing
// (linear) algorithm, estimate from a sample whether the data is clustered.
//
// Paper: each cell sent its maximum to its right neighbour, stepped through
// its own elements at evenly spaced intervals (a 1000-point sample, footnote
// 8) and counted the sampled elements below the received maximum, i.e. still
// overlapping the neighbour after bucketing; cells with 65 % or more such
// elements were problem cells, and more than two of them made the program
// switch to a more thorough algorithm.  Here one block takes the evenly
// spaced sample of the whole input, buckets each sampled key by the top bits
// of the sample's significant width (the bucketing an MSD plan would do),
// sorts the sample's buckets (they stand for the bucketed output), splits
// them into the output partitions ("cells") and applies the same test to
// each cell against its left neighbour's maximum bucket.  All integer
// arithmetic: the 65 % rule is 100 * overlap >= 65 * cell size.
#include <cstdint>

#include "rs_device.cuh"
#include "rs_internal.h"

namespace rs {
namespace {

constexpr int kSelectThreads = 1024;

__global__ void __launch_bounds__(kSelectThreads) select_kernel(const SelectArgs a) {
  __shared__ uint32_t b[kSelectThreads];
  __shared__ uint32_t s_max[kSelectThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t S = a.n < uint64_t(a.sample) ? uint32_t(a.n) : a.sample;
  uint32_t v = 0;
  if (uint32_t(tid) < S) {
    const uint64_t pos = (uint64_t(tid) * a.n) / S;  // floor(i * n / S)
    v = to_ordered(a.keys[pos], a.x);
  }
  // the sample's significant width
  uint32_t m = v;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) s_max[warp] = m;
  __syncthreads();
  if (warp == 0) {
    m = s_max[lane];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) s_max[0] = m;
  }
  __syncthreads();
  const uint32_t width = s_max[0] ? 32u - uint32_t(__clz(s_max[0])) : 0u;
  const uint32_t shift = width > a.bits ? width - a.bits : 0u;
  b[tid] = uint32_t(tid) < S ? (v >> shift) : 0xffffffffu;  // padding sorts last
  __syncthreads();
  // bitonic sort of the 1024 slots, ascending
  for (int k = 2; k <= kSelectThreads; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      const int p = tid ^ j;
      if (p > tid) {
        const uint32_t x = b[tid], y = b[p];
        const bool up = (tid & k) == 0;
        if ((x > y) == up) {
          b[tid] = y;
          b[p] = x;
        }
      }
      __syncthreads();
    }
  }
  // cell c >= 1 covers sample ranks [c*S/cells, (c+1)*S/cells)
  bool problem = false;
  const uint32_t c = uint32_t(tid);
  if (c >= 1 && c < a.cells) {
    const uint32_t lo = uint32_t((uint64_t(c) * S) / a.cells), hi = uint32_t((uint64_t(c + 1) * S) / a.cells);
    if (hi > lo && lo > 0) {  // an empty cell, or one with nothing to its left, has no overlap
      const uint32_t left_max = b[lo - 1];
      uint32_t over = 0;
      for (uint32_t r = lo; r < hi; ++r) over += b[r] <= left_max ? 1u : 0u;
      problem = 100u * over >= 65u * (hi - lo);
    }
  }
  const int count = __syncthreads_count(problem);
  if (tid == 0) {
    a.out[0] = uint32_t(count);
    a.out[1] = uint32_t(count) > a.max_problem ? 1u : 0u;
    a.out[2] = shift;
    a.out[3] = S;
  }
  if (a.buckets && uint32_t(tid) < S) a.buckets[tid] = b[tid];
}

}  // namespace

cudaError_t launch_select(const SelectArgs& a, cudaStream_t s) {
  if (a.sample < 1 || a.sample > uint32_t(kSelectThreads) || a.cells > uint32_t(kSelectThreads))
    return cudaErrorInvalidValue;
  select_kernel<<<1, kSelectThreads, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace rs
