// Stable merge of two sorted runs.
//
// Paper: the cleanup phase repaired the bucketed distribution by a
// merge-exchange between neighbouring cells, at whose heart two sorted lists
// are merged and each cell keeps its half (Sec. 3.4.2; later done in place,
// Sec. 4.6).  On the GPU a merge of two
// sorted runs A and B splits the output into tiles of TILE elements; the
// tile boundaries are placed on the merge path (for output position d, the
// number of elements of A among the first d outputs), found by a binary
// search per boundary; each block then loads its slices of A and B into
// shared memory, every thread finds its own start on the path inside the
// tile and merges ITEMS outputs in registers, and the tile leaves through
// shared memory in coalesced stores.  Equal keys keep A's before B's
// (stable), keys of every kind compare through the order map of KeyXform.
#include <cuda_runtime.h>

#include "rs_device.cuh"
#include "rs_internal.h"

namespace rs {

namespace {

// ITEMS is odd: a thread's ITEMS consecutive outputs start ITEMS words after
// its neighbour's, so a warp's staging stores fall on 32 different banks.
constexpr int kMergeThreads = 256;
// tile shapes 1..4; key+payload tiles of 23 items take
// 47 KB of static shared memory, the most a block can declare statically
constexpr int kMergeItemsChoice[] = {15, 11, 23, 19};
__device__ __forceinline__ uint32_t slot(uint32_t i) { return i; }

// Elements of A among the first d outputs of the stable merge of a[0, na)
// and b[0, nb): the smallest i with A[i] coming after B[d - i - 1], where A
// comes first on equal keys.  `at(x, k)` reads element k of run x mapped.
template <class F>
__device__ __forceinline__ uint32_t path_split(F at, uint32_t na, uint32_t nb, uint32_t d) {
  uint32_t lo = d > nb ? d - nb : 0u, hi = d < na ? d : na;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (at(0, mid) <= at(1, d - mid - 1)) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// One warp per tile boundary: the same search as path_split, but each
// round probes 32 points of the remaining range at once (a ballot finds
// where "A first" turns false), so a boundary costs about log_33 of the range
// rounds of dependent loads instead of log_2.
template <bool XF>
__global__ void __launch_bounds__(256) merge_split_kernel(const MergeArgs m) {
  const uint32_t k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const uint32_t total = m.na + m.nb;
  const uint32_t tiles = (total + m.tile - 1) / m.tile;
  if (k > tiles) return;  // whole warps leave together
  const uint64_t d64 = uint64_t(k) * m.tile;
  const uint32_t d = d64 < total ? uint32_t(d64) : total;
  // true when A[i] comes before B[d - i - 1], i.e. the answer is above i
  auto a_first = [&](uint32_t i) {
    if constexpr (XF) return to_ordered(m.a[i], m.x) <= to_ordered(m.b[d - i - 1], m.x);
    else return m.a[i] <= m.b[d - i - 1];
  };
  uint32_t lo = d > m.nb ? d - m.nb : 0u, hi = d < m.na ? d : m.na;  // answer in [lo, hi]
  while (hi - lo > 32) {
    const uint64_t len = hi - lo;
    const uint32_t i = lo + uint32_t(len * (lane + 1) / 33);  // in [lo, hi)
    const uint32_t t = __ballot_sync(0xffffffffu, a_first(i));
    const uint32_t f = __popc(t);  // probes that are true come first (sorted runs)
    const uint32_t i_prev = lo + uint32_t(len * f / 33);        // probe f - 1 (f >= 1)
    const uint32_t i_f = lo + uint32_t(len * (f + 1) / 33);     // probe f (f <= 31)
    const uint32_t nlo = f == 0 ? lo : i_prev + 1;
    const uint32_t nhi = f == 32 ? hi : i_f;
    lo = nlo;
    hi = nhi > nlo ? nhi : nlo;
  }
  const bool probe = lo + lane < hi && a_first(lo + lane);
  const uint32_t t = __ballot_sync(0xffffffffu, probe);
  if (lane == 0) m.split[k] = lo + __popc(t);
}

template <bool PAIRS, bool XF, int kMergeItems>
__global__ void __launch_bounds__(kMergeThreads) merge_tile_kernel(const MergeArgs m) {
  constexpr int kMergeTile = kMergeThreads * kMergeItems;
  __shared__ uint32_t s_key[kMergeTile];
  __shared__ uint32_t s_val[PAIRS ? kMergeTile : 1];
  const uint32_t total = m.na + m.nb;
  const uint32_t t = blockIdx.x, tid = threadIdx.x;
  const uint32_t d0 = t * kMergeTile;
  const uint32_t d1 = total - d0 < uint32_t(kMergeTile) ? total : d0 + kMergeTile;
  const uint32_t i0 = m.split[t], i1 = m.split[t + 1];
  // On sorted runs the path is monotone: i0 <= i1 and i1 - i0 <= d1 - d0.
  // Runs that are not sorted can break that; the tile is then not written
  // and the error word is raised instead of reading past the slices.
  if (i1 < i0 || i1 - i0 > d1 - d0) {
    if (tid == 0) atomicOr(m.err, kErrBounds);
    return;
  }
  const uint32_t j0 = d0 - i0, j1 = d1 - i1;
  const uint32_t la = i1 - i0, lb = j1 - j0;  // la + lb = d1 - d0 <= TILE
  // this tile's slices of A then B, mapped, side by side (all of a
  // thread's loads are issued before the first store)
  {
    uint32_t ld[kMergeItems], lv[PAIRS ? kMergeItems : 1];
#pragma unroll
    for (int q = 0; q < kMergeItems; ++q) {
      const uint32_t e = tid + q * kMergeThreads;
      if (e < la + lb) {
        const bool from_a = e < la;
        ld[q] = from_a ? m.a[i0 + e] : m.b[j0 + e - la];
        if constexpr (PAIRS) lv[q] = from_a ? m.va[i0 + e] : m.vb[j0 + e - la];
      }
    }
#pragma unroll
    for (int q = 0; q < kMergeItems; ++q) {
      const uint32_t e = tid + q * kMergeThreads;
      if (e < la + lb) {
        s_key[slot(e)] = XF ? to_ordered(ld[q], m.x) : ld[q];
        if constexpr (PAIRS) s_val[slot(e)] = lv[q];
      }
    }
  }
  __syncthreads();
  // this thread's ITEMS outputs start on the path at diagonal tid * ITEMS
  const uint32_t dt = tid * kMergeItems < la + lb ? tid * kMergeItems : la + lb;
  auto at = [&](int x, uint32_t i) { return s_key[slot(x == 0 ? i : la + i)]; };
  uint32_t ia = path_split(at, la, lb, dt), ib = dt - ia;
  // the heads of both slices stay in registers: one shared-memory read per
  // output (an exhausted slice reads as "comes last")
  uint32_t ha = ia < la ? s_key[slot(ia)] : 0u, hb = ib < lb ? s_key[slot(la + ib)] : 0u;
  uint32_t key[kMergeItems], src[kMergeItems];
#pragma unroll
  for (int q = 0; q < kMergeItems; ++q) {
    const bool take_a = ia < la && (ib >= lb || ha <= hb);
    src[q] = take_a ? ia : la + ib;  // position in the shared slices
    key[q] = take_a ? ha : hb;
    if (take_a) {
      ++ia;
      ha = ia < la ? s_key[slot(ia)] : 0u;
    } else {
      ++ib;
      hb = ib < lb ? s_key[slot(la + ib)] : 0u;
    }
  }
  uint32_t val[PAIRS ? kMergeItems : 1];
  if constexpr (PAIRS) {
#pragma unroll
    for (int q = 0; q < kMergeItems; ++q) val[q] = s_val[slot(src[q] < la + lb ? src[q] : 0)];
  }
  __syncthreads();  // the slices are consumed; the tile is staged in their place
#pragma unroll
  for (int q = 0; q < kMergeItems; ++q) {
    const uint32_t o = tid * kMergeItems + q;
    if (o < la + lb) {
      s_key[slot(o)] = key[q];
      if constexpr (PAIRS) s_val[slot(o)] = val[q];
    }
  }
  __syncthreads();
  for (uint32_t e = tid; e < la + lb; e += kMergeThreads) {
    m.out[d0 + e] = XF ? from_ordered(s_key[slot(e)], m.x) : s_key[slot(e)];
    if constexpr (PAIRS) m.vout[d0 + e] = s_val[slot(e)];
  }
}

template <int ITEMS>
void launch_tiles(const MergeArgs& m, unsigned tiles, cudaStream_t s) {
  const bool xf = !is_identity(m.x);
  if (m.vout) {
    if (xf) merge_tile_kernel<true, true, ITEMS><<<tiles, kMergeThreads, 0, s>>>(m);
    else merge_tile_kernel<true, false, ITEMS><<<tiles, kMergeThreads, 0, s>>>(m);
  } else {
    if (xf) merge_tile_kernel<false, true, ITEMS><<<tiles, kMergeThreads, 0, s>>>(m);
    else merge_tile_kernel<false, false, ITEMS><<<tiles, kMergeThreads, 0, s>>>(m);
  }
}

}  // namespace

// Outputs per tile of merge tile shape `shape` (1-based), or 0 if there is
// no such shape.  Shape 0 picks the measured default: 23 items per thread for
// keys, 19 with payloads (GB300, two runs of 2^26: 326 and 503 us).
uint32_t merge_tile_keys(uint32_t shape, bool pairs) {
  const uint32_t idx = shape == 0 ? (pairs ? 3u : 2u) : shape - 1;
  if (idx >= sizeof(kMergeItemsChoice) / sizeof(kMergeItemsChoice[0])) return 0;
  return uint32_t(kMergeThreads * kMergeItemsChoice[idx]);
}

cudaError_t launch_merge(const MergeArgs& m, cudaStream_t s) {
  const uint32_t total = m.na + m.nb;
  const uint32_t tiles = (total + m.tile - 1) / m.tile;
  const unsigned sgrid = (tiles + 1 + 7) / 8;  // a warp per boundary
  if (!is_identity(m.x)) merge_split_kernel<true><<<sgrid, 256, 0, s>>>(m);
  else merge_split_kernel<false><<<sgrid, 256, 0, s>>>(m);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || tiles == 0) return e;
  switch (m.tile / kMergeThreads) {
    case 15: launch_tiles<15>(m, tiles, s); break;
    case 11: launch_tiles<11>(m, tiles, s); break;
    case 23: launch_tiles<23>(m, tiles, s); break;
    case 19: launch_tiles<19>(m, tiles, s); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace rs
