// The MSD plan's bucketing: keys distributed by their top bits into 2^14
// buckets in one pass, with exact per-(chunk, bucket) offsets computed from
// one counting read; each bucket then goes through the segmented pipeline
// (one-block local sort of the low bits for buckets that fit, tiled passes
// for the others).
//
// Paper: the bucketing phase of Sec. 3.2 (each cell counts its elements per
// bucket, the cumulative totals give where each bucket goes, the elements are
// distributed) followed by the local radix sort of each cell's range (the
// revised pipeline of Sec. 4.6).  The paper used 4096 and then 8192 buckets
// (Sec. 3.2, Sec. 4.7); here the bucket is the key's bits 18-31, which gives
// 8192 buckets of about 8K keys for 2^26 uniform 31-bit keys and 16384 for
// full 32-bit keys, each within the 16,384-key local sort.  The paper's
// cells distributed with approximate offsets and repaired them later
// (Sec. 3.2, Sec. 3.4); here each of C chunks (one per block) has its exact
// offset for every bucket: per-chunk bucket counts, an exclusive scan down
// each bucket's column of chunks, and the bucket bases.
//
// Keys only: inside a chunk, a key takes its position in its bucket by a
// shared-memory atomic on the chunk's cursor for that bucket.  The order of
// keys inside a bucket is then not the input order, which does not matter:
// every bucket is sorted on all its remaining bits afterwards and equal keys
// are indistinguishable.  (Key+payload sorts must keep equal keys in input
// order and take the bucketing as two stable LSD passes over bits 18-24 and
// 25-31 instead; api.cu.)
#include <cstdint>

#include "rs_device.cuh"
#include "rs_internal.h"

namespace rs {
namespace {

constexpr int kMsdThreads = 1024;
constexpr int kMsdBins = 1 << (32 - kMsdShift);

// The keys of chunk c: [c * len, min(n, (c + 1) * len)).
struct Chunk {
  uint64_t lo, hi;
};
__device__ __forceinline__ Chunk chunk_of(uint64_t n, uint32_t chunks, uint32_t c) {
  const uint64_t len = (n + chunks - 1) / chunks;
  const uint64_t lo = uint64_t(c) * len;
  const uint64_t hi = lo + len < n ? lo + len : n;
  return Chunk{lo < n ? lo : n, hi};
}

// Counts of the chunk's keys per bucket -> hist[c][bucket].
__global__ void __launch_bounds__(kMsdThreads, 1) msd_count_kernel(const MsdArgs a) {
  extern __shared__ __align__(16) uint32_t sh[];  // [kMsdBins]
  for (int i = threadIdx.x; i < kMsdBins; i += kMsdThreads) sh[i] = 0u;
  __syncthreads();
  const Chunk ch = chunk_of(a.n, a.chunks, blockIdx.x);
  const uint32_t base = uint32_t(__cvta_generic_to_shared(sh));
  constexpr int U = 8;
  uint64_t i = ch.lo + threadIdx.x;
  for (; i + uint64_t(U - 1) * kMsdThreads < ch.hi; i += uint64_t(U) * kMsdThreads) {
    uint32_t k[U];
#pragma unroll
    for (int u = 0; u < U; ++u) k[u] = ld_stream(a.keys + i + u * kMsdThreads);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint32_t d = to_ordered(k[u], a.x) >> kMsdShift;
      asm volatile("red.shared.add.u32 [%0], 1;" ::"r"(base + 4u * d) : "memory");
    }
  }
  for (; i < ch.hi; i += kMsdThreads) {
    const uint32_t d = to_ordered(a.keys[i], a.x) >> kMsdShift;
    asm volatile("red.shared.add.u32 [%0], 1;" ::"r"(base + 4u * d) : "memory");
  }
  __syncthreads();
  uint32_t* row = a.hist + size_t(blockIdx.x) * kMsdBins;
  for (int b = threadIdx.x; b < kMsdBins; b += kMsdThreads) row[b] = sh[b];
}

// Per bucket: exclusive scan down its column of chunks (in place), and the
// bucket's total.
__global__ void __launch_bounds__(256) msd_colscan_kernel(const MsdArgs a) {
  const uint32_t d = blockIdx.x * 256 + threadIdx.x;
  if (d >= uint32_t(kMsdBins)) return;
  uint32_t run = 0;
  for (uint32_t c = 0; c < a.chunks; ++c) {
    uint32_t* p = a.hist + size_t(c) * kMsdBins + d;
    const uint32_t v = *p;
    *p = run;
    run += v;
  }
  a.totals[d] = run;
}

// Bucket bases (exclusive scan of the totals, in place) and the buckets as
// segments: seg_off[b] = base of bucket b, seg_off[kMsdBins] = n.
__global__ void __launch_bounds__(1024) msd_basescan_kernel(const MsdArgs a) {
  __shared__ uint32_t s_warp[32];
  __shared__ uint32_t s_carry, s_total;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (int c0 = 0; c0 < kMsdBins; c0 += 1024) {
    const int d = c0 + threadIdx.x;
    const uint32_t v = a.totals[d];
    const uint32_t ex = block_exclusive_sum<1024>(v, s_warp, &s_total);  // ends with a barrier
    const uint32_t b = s_carry + ex;
    a.totals[d] = b;
    a.seg_off[d] = b;
    __syncthreads();  // every thread has read s_carry and s_total
    if (threadIdx.x == 0) s_carry += s_total;
    __syncthreads();
  }
  if (threadIdx.x == 0) a.seg_off[kMsdBins] = a.n;
}

// The distribution: each key to base[bucket] + (earlier chunks' keys of the
// bucket) + its turn among this chunk's keys of the bucket (a shared-memory
// atomic).  Keys are written in their order-mapped form (the local phase
// maps them back).  An index outside [0, n) is skipped and reported.
__global__ void __launch_bounds__(kMsdThreads, 1) msd_scatter_kernel(const MsdArgs a) {
  extern __shared__ __align__(16) uint32_t sh[];  // [kMsdBins] cursors
  const uint32_t* colex = a.hist + size_t(blockIdx.x) * kMsdBins;
  for (int b = threadIdx.x; b < kMsdBins; b += kMsdThreads) sh[b] = a.totals[b] + colex[b];
  __syncthreads();
  const Chunk ch = chunk_of(a.n, a.chunks, blockIdx.x);
  const uint32_t base = uint32_t(__cvta_generic_to_shared(sh));
  bool oob = false;
  auto put = [&](uint32_t k) {
    const uint32_t m = to_ordered(k, a.x);
    uint32_t pos;
    asm volatile("atom.shared.add.u32 %0, [%1], 1;" : "=r"(pos) : "r"(base + 4u * (m >> kMsdShift)) : "memory");
    if (pos < a.n) a.out[pos] = m;
    else oob = true;
  };
  constexpr int U = 8;
  uint64_t i = ch.lo + threadIdx.x;
  for (; i + uint64_t(U - 1) * kMsdThreads < ch.hi; i += uint64_t(U) * kMsdThreads) {
    uint32_t k[U];
#pragma unroll
    for (int u = 0; u < U; ++u) k[u] = ld_stream(a.keys + i + u * kMsdThreads);
#pragma unroll
    for (int u = 0; u < U; ++u) put(k[u]);
  }
  for (; i < ch.hi; i += kMsdThreads) put(a.keys[i]);
  if (oob) atomicOr(a.err, kErrBounds);
}

}  // namespace

size_t msd_smem() { return size_t(kMsdBins) * 4; }
const void* msd_count_func() { return reinterpret_cast<const void*>(&msd_count_kernel); }
const void* msd_scatter_func() { return reinterpret_cast<const void*>(&msd_scatter_kernel); }

cudaError_t launch_msd_count(const MsdArgs& a, cudaStream_t s) {
  msd_count_kernel<<<a.chunks, kMsdThreads, msd_smem(), s>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_msd_scan(const MsdArgs& a, cudaStream_t s) {
  msd_colscan_kernel<<<(kMsdBins + 255) / 256, 256, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  msd_basescan_kernel<<<1, 1024, 0, s>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_msd_scatter(const MsdArgs& a, cudaStream_t s) {
  msd_scatter_kernel<<<a.chunks, kMsdThreads, msd_smem(), s>>>(a);
  return cudaGetLastError();
}

}  // namespace rs
