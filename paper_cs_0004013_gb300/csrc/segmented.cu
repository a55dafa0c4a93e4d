// Many independent sorts in one pipeline: the segments of a concatenated
// array, planned on the device.
//
// Paper: each segment is sorted by the same radix distribution as a whole
// array (Sec. 3.2, Sec. 3.3.1).  The split into small segments sorted
// entirely inside one block and large ones sorted by tiled passes mirrors
// the paper's two levels: bucketing into per-cell ranges, then a local
// radix sort of each cell's data (Sec. 3, revised pipeline of Sec. 4.6).
// The MSD plan uses the same pipeline on the buckets of the top digit.
//
// Launch sequence (all on one stream, sizes only known on the device are
// handled by persistent grid-stride loops):
//   seg_plan      one block: classify segments (empty / tiny / small /
//                 large), list them, number the tiles of large segments;
//   seg_hist      per large tile: digit histograms into the segment's
//                 arrays; clears the tile's status row;
//   seg_scan      per large segment and digit: exclusive scan;
//   seg_pass x P  onesweep passes over the large tiles, lookback confined to
//                 the tile's own segment;
//   local_sort    one block per tiny / small segment: every digit sorted
//                 in shared memory, written once.
#include <cuda_runtime.h>

#include "onesweep.cuh"
#include "rs_device.cuh"
#include "rs_internal.h"

namespace rs {

namespace {

// ---------------------------------------------------------------- planning
__global__ void __launch_bounds__(1024) seg_plan_kernel(const SegPlanArgs a) {
  __shared__ uint32_t s_warp[32];
  __shared__ uint32_t s_tot[4];
  uint32_t carry_l = 0, carry_s = 0, carry_t = 0, carry_tiles = 0;
  const uint32_t n_chunks = (a.num_segs + 1023u) / 1024u;
  for (uint32_t c = 0; c < n_chunks; ++c) {
    const uint32_t s = c * 1024u + threadIdx.x;
    uint64_t m = 0;
    if (s < a.num_segs) m = a.seg_off[s + 1] - a.seg_off[s];
    const bool valid = s < a.num_segs && m > 0;
    const bool tiny = valid && m <= a.tiny_max;
    const bool small = valid && !tiny && m <= a.small_max;
    const bool large = valid && m > a.small_max;
    const uint32_t nt = large ? uint32_t((m + a.tile - 1) / a.tile) : 0u;
    const uint32_t el = block_exclusive_sum<1024>(large ? 1u : 0u, s_warp, &s_tot[0]);
    const uint32_t es = block_exclusive_sum<1024>(small ? 1u : 0u, s_warp, &s_tot[1]);
    const uint32_t et = block_exclusive_sum<1024>(tiny ? 1u : 0u, s_warp, &s_tot[2]);
    const uint32_t ex = block_exclusive_sum<1024>(nt, s_warp, &s_tot[3]);
    if (large) {
      a.large_seg[carry_l + el] = s;
      a.tile_prefix[carry_l + el] = carry_tiles + ex;
    }
    if (small) a.small_seg[carry_s + es] = s;
    if (tiny) a.tiny_seg[carry_t + et] = s;
    carry_l += s_tot[0];
    carry_s += s_tot[1];
    carry_t += s_tot[2];
    carry_tiles += s_tot[3];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    a.tile_prefix[carry_l] = carry_tiles;
    a.counts[SEG_NUM_LARGE] = carry_l;
    a.counts[SEG_NUM_SMALL] = carry_s;
    a.counts[SEG_NUM_TINY] = carry_t;
    a.counts[SEG_NUM_TILES] = carry_tiles;
  }
}

// Index of the large segment holding large tile t (the last i with
// tile_prefix[i] <= t).
__device__ __forceinline__ uint32_t find_segment(const uint32_t* tile_prefix, uint32_t num_large, uint32_t t) {
  uint32_t lo = 0, hi = num_large;  // invariant: tile_prefix[lo] <= t < tile_prefix[hi]
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (tile_prefix[mid] <= t) lo = mid;
    else hi = mid;
  }
  return lo;
}

// -------------------------------------------------------------- histograms
// Each block takes a contiguous run of large tiles, so that consecutive
// tiles usually belong to the same segment.  Every lane counts into its own
// copy of the digit histograms, laid out [digit][bin][lane] so that lane l
// only touches shared-memory bank l (no atomic conflicts whatever the
// digits); the copies are summed into the segment's global arrays when the
// run moves on to the next segment, and at the end.  Also writes each
// tile's job entry and clears its chained-scan status row.  The digits are
// the key's low num_digits bytes (the launcher checks): each is taken with
// one byte permute and counted with one shared-memory reduction on a 32-bit
// shared address (the count loop is bound by integer instructions).
template <int THREADS, bool XF>
__global__ void __launch_bounds__(THREADS, 1) seg_hist_kernel(const SegHistArgs a) {
  extern __shared__ __align__(16) uint32_t sh[];  // [num_digits][256][32]
  const uint32_t num_large = a.counts[SEG_NUM_LARGE], total = a.counts[SEG_NUM_TILES];
  const int nd = a.num_digits;
  const int tid = threadIdx.x, lane = tid & 31;
  const uint32_t per = (total + gridDim.x - 1) / gridDim.x;
  const uint32_t t_begin = blockIdx.x * per;
  const uint32_t t_end = t_begin + per < total ? t_begin + per : total;
  if (t_begin >= t_end) return;  // uniform across the block
  for (int i = tid; i < nd * 256 * 32; i += THREADS) sh[i] = 0u;
  // this lane's copy of bin 0 of digit 0; (digit j, bin b) is 32 KiB * j + 128 * b bytes further
  const uint32_t lane_base = uint32_t(__cvta_generic_to_shared(sh)) + uint32_t(lane) * 4u;
  const KeyXform xf = a.xform;
  // sums a segment's lane copies into its global histograms and zeroes them;
  // each thread owns whole (digit, bin) rows and starts at its own lane, so
  // that a warp's reads spread over all banks
  auto flush = [&](uint32_t li) {
    __syncthreads();
    uint32_t* h = a.seg_hist + size_t(li) * nd * 256;
    for (int r = tid; r < nd * 256; r += THREADS) {
      uint32_t sum = 0;
#pragma unroll 8
      for (int k = 0; k < 32; ++k) {
        uint32_t* c = &sh[r * 32 + ((k + lane) & 31)];
        sum += *c;
        *c = 0u;
      }
      if (sum) atomicAdd(&h[r], sum);
    }
    __syncthreads();
  };
  // the segment of the run's first tile; later ones are found by stepping
  uint32_t li = find_segment(a.tile_prefix, num_large, t_begin);
  uint32_t first = a.tile_prefix[li], next = a.tile_prefix[li + 1];
  uint32_t s = a.large_seg[li];
  uint64_t seg_start = a.seg_off[s], seg_end = a.seg_off[s + 1];
  __syncthreads();
  // The block's tiles of one segment form one contiguous key range: it is
  // counted in one sweep (whatever the tile size, every sweep iteration but
  // the last keeps all loads busy), then the tiles' job entries are written
  // and their status rows cleared.
  uint32_t t = t_begin;
  while (t < t_end) {
    if (t >= next) {  // uniform: every thread steps the same way
      flush(li);
      do {
        ++li;
        first = next;
        next = a.tile_prefix[li + 1];
      } while (t >= next);
      s = a.large_seg[li];
      seg_start = a.seg_off[s];
      seg_end = a.seg_off[s + 1];
    }
    const uint32_t run_end = next < t_end ? next : t_end;  // this segment's tiles in the block's range
    const uint64_t rs = seg_start + uint64_t(t - first) * a.tile;
    const uint64_t re_full = seg_start + uint64_t(run_end - first) * a.tile;
    const uint64_t re = re_full < seg_end ? re_full : seg_end;
    for (uint32_t u = t + tid; u < run_end; u += THREADS) {
      const uint64_t start = seg_start + uint64_t(u - first) * a.tile;
      const uint64_t end = start + a.tile < seg_end ? start + a.tile : seg_end;
      a.jobs[u] = SegTileJob{start, uint32_t(end - start), first, uint32_t(seg_start), uint32_t(seg_end), li, 0u};
    }
    // the tiles' chained-scan status rows start out "not ready"
    for (size_t z = tid; z < size_t(run_end - t) * 256; z += THREADS) a.status[size_t(t) * 256 + z] = 0u;
    // eight loads in flight per thread before the counting (measured faster
    // than two 16-byte vectors per thread)
    for (uint64_t i0 = rs + tid; i0 < re; i0 += 8 * THREADS) {
      uint32_t k[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const uint64_t i = i0 + uint64_t(u) * THREADS;
        k[u] = i < re ? ld_stream(a.keys + i) : 0u;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (i0 + uint64_t(u) * THREADS >= re) break;
        const uint32_t kk = XF ? to_ordered(k[u], xf) : k[u];
#pragma unroll
        for (int j = 0; j < kMaxDigits; ++j) {
          if (j < nd) {
            const uint32_t b = __byte_perm(kk, 0u, 0x4440u + uint32_t(j));
            const uint32_t addr = lane_base + uint32_t(j * 256 * 32 * 4) + b * 128u;
            asm volatile("red.shared.add.u32 [%0], 1;" ::"r"(addr) : "memory");
          }
        }
      }
    }
    t = run_end;
  }
  flush(li);
}

__global__ void __launch_bounds__(256) seg_scan_kernel(const SegScanArgs a) {
  __shared__ uint32_t s_warp[32];
  const uint32_t num_large = a.counts[SEG_NUM_LARGE];
  for (uint32_t li = blockIdx.x; li < num_large; li += gridDim.x) {
    for (int j = 0; j < a.num_digits; ++j) {
      const size_t at = (size_t(li) * a.num_digits + j) * 256 + threadIdx.x;
      const uint32_t v = a.seg_hist[at];
      a.seg_bases[at] = block_exclusive_sum<256>(v, s_warp);
    }
  }
}

// ------------------------------------------------------------ tiled passes
template <int THREADS, int ITEMS, bool PAIRS, int MINB>
__global__ void __launch_bounds__(THREADS, MINB) seg_pass_kernel(const SegPassArgs a) {
  using L = OnesweepLayout<8, THREADS, ITEMS, PAIRS>;
  extern __shared__ __align__(16) unsigned char smem[];
  const uint32_t total = a.counts[SEG_NUM_TILES];
  for (;;) {
    const uint32_t t = begin_tile<8, THREADS, ITEMS, PAIRS>(a.tile_counter, smem);
    if (t >= total) return;  // uniform across the block
    const SegTileJob jb = a.jobs[t];
    TileJob job;
    job.tile = t;
    job.first = jb.first;
    job.base = jb.base;
    job.valid = jb.valid;
    job.out_start = jb.out_start;
    job.out_end = jb.out_end;
    job.bases = a.seg_bases + (size_t(jb.li) * a.num_digits + a.pass) * 256;
    const PairIO none{nullptr, nullptr, 0, 0u, KeyXform64{0u, 0u, 0u}, 0, nullptr, nullptr, 0u};
    onesweep_tile<8, THREADS, ITEMS, PAIRS ? 1 : 0, uint32_t, false>(job, a.kin, a.kout, a.vin, a.vout, nullptr,
                                                                      nullptr, none, a.shift, a.width, a.status,
                                                                      a.parity, a.err, a.xin, a.xout, smem);
    __syncthreads();  // the next tile reuses shared memory
  }
}

// ------------------------------------------------------ one-block local sort
template <int THREADS, int ITEMS, bool PAIRS>
struct LocalLayout {
  static constexpr int WARPS = THREADS / 32;
  static constexpr int TILE = THREADS * ITEMS;
  static constexpr size_t MASK_BYTES = size_t(WARPS) * kMaskSlots * 4;
  static constexpr size_t CNT_BYTES = size_t(WARPS) * 256 * 2;
  static constexpr size_t OFF_BUF = MASK_BYTES + CNT_BYTES;
  static constexpr size_t BUF_BYTES = size_t(TILE) * 4 * (PAIRS ? 2 : 1);
  static constexpr size_t OFF_WARP = OFF_BUF + BUF_BYTES;
  static constexpr size_t SMEM = OFF_WARP + 32 * 4;
  static_assert(THREADS >= 256, "one thread per 8-bit digit in the scan");
  static_assert((MASK_BYTES + CNT_BYTES) % 16 == 0, "tables are cleared in 16-byte units");
};

// Sorts each listed segment (at most THREADS * ITEMS keys) by every digit
// of the plan, least significant first, entirely in shared memory: per
// digit a stable warp rank (the same lane-mask tables as the tiled pass),
// per-digit tile offsets, and a scatter into the staging buffer, which the
// next digit reads back.  Keys past the segment's end act as 0xFFFFFFFF and
// stay behind every real key.  Writes src -> dst once.
template <int THREADS, int ITEMS, bool PAIRS>
__global__ void __launch_bounds__(THREADS, 1) local_sort_kernel(const LocalArgs a) {
  using L = LocalLayout<THREADS, ITEMS, PAIRS>;
  constexpr int TILE = L::TILE, WARPS = L::WARPS;
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* s_mask = reinterpret_cast<uint32_t*>(smem);
  uint16_t* s_cnt = reinterpret_cast<uint16_t*>(smem + L::MASK_BYTES);
  uint32_t* s_buf = reinterpret_cast<uint32_t*>(smem + L::OFF_BUF);
  uint32_t* s_warp = reinterpret_cast<uint32_t*>(smem + L::OFF_WARP);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // a listed set of segments, or (list == null) the one array [0, single_n)
  const uint32_t count = a.list ? *a.count : 1u;
  for (uint32_t k = blockIdx.x; k < count; k += gridDim.x) {
    const uint32_t s = a.list ? a.list[k] : 0u;
    const uint64_t start = a.list ? a.seg_off[s] : 0u;
    const uint32_t m = a.list ? uint32_t(a.seg_off[s + 1] - start) : a.single_n;
    uint32_t key[ITEMS], val[PAIRS ? ITEMS : 1];
    const uint32_t wofs = uint32_t(warp) * 32 * ITEMS + lane;
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      const uint32_t i = wofs + j * 32;
      key[j] = i < m ? to_ordered(a.kin[start + i], a.xin) : 0xffffffffu;
      if constexpr (PAIRS) val[j] = i < m ? a.vin[start + i] : 0u;
    }
    for (int p = 0; p < a.num_digits; ++p) {
      const uint32_t shift = a.dig[p].shift, width = a.dig[p].width;
      uint4* c4 = reinterpret_cast<uint4*>(smem);
      for (int i = tid; i < int(L::OFF_BUF / 16); i += THREADS) c4[i] = make_uint4(0u, 0u, 0u, 0u);
      __syncthreads();
      uint32_t rk[(ITEMS + 1) / 2];
      warp_rank<8, ITEMS>(key, shift, width, s_mask + warp * kMaskSlots, s_cnt + warp * 256, rk);
      __syncthreads();
      // per digit (threads 0..255): total over warps, exclusive over digits,
      // then exclusive (digit, warp) offsets
      uint32_t tot = 0;
      if (tid < 256)
        for (int wi = 0; wi < WARPS; ++wi) tot += s_cnt[wi * 256 + tid];
      const uint32_t excl = block_exclusive_sum<THREADS>(tid < 256 ? tot : 0u, s_warp);
      if (tid < 256) {
        uint32_t run = excl;
        for (int wi = 0; wi < WARPS; ++wi) {
          const uint32_t v = s_cnt[wi * 256 + tid];
          s_cnt[wi * 256 + tid] = uint16_t(run);
          run += v;
        }
      }
      __syncthreads();
#pragma unroll
      for (int j = 0; j < ITEMS; ++j) {
        const uint32_t pos = ((rk[j >> 1] >> (16 * (j & 1))) & 0xffffu) + s_cnt[warp * 256 + digit_of(key[j], shift, width)];
        s_buf[pos] = key[j];
        if constexpr (PAIRS) s_buf[TILE + pos] = val[j];
      }
      __syncthreads();
#pragma unroll
      for (int j = 0; j < ITEMS; ++j) {
        key[j] = s_buf[wofs + j * 32];
        if constexpr (PAIRS) val[j] = s_buf[TILE + wofs + j * 32];
      }
      __syncthreads();
    }
    // the staging buffer holds the sorted segment (then the padding)
    for (uint32_t i = tid; i < m; i += THREADS) {
      a.kout[start + i] = from_ordered(s_buf[i], a.xout);
      if constexpr (PAIRS) a.vout[start + i] = s_buf[TILE + i];
    }
    __syncthreads();
  }
}

// Bucket offsets of an MSD plan: the exclusive scan of the top digit as
// segment offsets (uint64), the last one being n.
__global__ void bases_to_offsets_kernel(const uint32_t* bases, uint32_t num, uint64_t n, uint64_t* seg_off) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < num) seg_off[i] = bases[i];
  if (i == num) seg_off[i] = n;
}

template <int THREADS, int ITEMS, bool PAIRS, int MINB>
cudaError_t launch_seg_pass(const SegPassArgs& a, unsigned grid, cudaStream_t s) {
  using L = OnesweepLayout<8, THREADS, ITEMS, PAIRS>;
  seg_pass_kernel<THREADS, ITEMS, PAIRS, MINB><<<grid, THREADS, L::SMEM, s>>>(a);
  return cudaGetLastError();
}

template <int THREADS, int ITEMS, bool PAIRS>
cudaError_t launch_local(const LocalArgs& a, unsigned grid, cudaStream_t s) {
  using L = LocalLayout<THREADS, ITEMS, PAIRS>;
  local_sort_kernel<THREADS, ITEMS, PAIRS><<<grid, THREADS, L::SMEM, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

// Tiled passes over large segments, 8-bit digits.  Shape 0: 512 x 16 tiles
// (keys and key+payload); shape 1: 512 x 24 for keys, 512 x 22 for
// key+payload; shape 2 (the default): 384 x 20 for both, three blocks per SM
// (the batch of 1774 key+payload arrays: 47.7 Gkeys/s against 47.0; 384 x 24
// spills in the persistent loop and takes 39.6).
constexpr int kSegThreads = 512, kSegItemsKeys = 24, kSegItemsPairs = 22, kSegItemsSmall = 16;
constexpr int kSegThreads3 = 384, kSegItems3 = 20;
// Local sorts: tiny segments <= 256 x 16 keys, small ones <= 1024 x 16 keys.
constexpr int kTinyThreads = 256, kSmallThreads = 1024, kLocalItems = 16;
// Segment histograms: one 1024-thread block per SM (lane copies of up to
// four digits take 128 KiB).
constexpr int kSegHistThreads = 1024;

const SegKernels* seg_kernels() {
  static const SegKernels k = {
      {uint32_t(kSegThreads * kSegItemsSmall), uint32_t(kSegThreads * kSegItemsKeys),
       uint32_t(kSegThreads3 * kSegItems3)},
      {uint32_t(kSegThreads * kSegItemsSmall), uint32_t(kSegThreads * kSegItemsPairs),
       uint32_t(kSegThreads3 * kSegItems3)},
      uint32_t(kTinyThreads * kLocalItems),
      uint32_t(kSmallThreads * kLocalItems),
      {2u, 2u, 3u},
      {OnesweepLayout<8, kSegThreads, kSegItemsSmall, 0>::SMEM, OnesweepLayout<8, kSegThreads, kSegItemsKeys, 0>::SMEM,
       OnesweepLayout<8, kSegThreads3, kSegItems3, 0>::SMEM},
      {OnesweepLayout<8, kSegThreads, kSegItemsSmall, 1>::SMEM, OnesweepLayout<8, kSegThreads, kSegItemsPairs, 1>::SMEM,
       OnesweepLayout<8, kSegThreads3, kSegItems3, 1>::SMEM},
      LocalLayout<kTinyThreads, kLocalItems, false>::SMEM,
      LocalLayout<kTinyThreads, kLocalItems, true>::SMEM,
      LocalLayout<kSmallThreads, kLocalItems, false>::SMEM,
      LocalLayout<kSmallThreads, kLocalItems, true>::SMEM,
      {reinterpret_cast<const void*>(&seg_pass_kernel<kSegThreads, kSegItemsSmall, false, 2>),
       reinterpret_cast<const void*>(&seg_pass_kernel<kSegThreads, kSegItemsKeys, false, 2>),
       reinterpret_cast<const void*>(&seg_pass_kernel<kSegThreads3, kSegItems3, false, 3>)},
      {reinterpret_cast<const void*>(&seg_pass_kernel<kSegThreads, kSegItemsSmall, true, 2>),
       reinterpret_cast<const void*>(&seg_pass_kernel<kSegThreads, kSegItemsPairs, true, 2>),
       reinterpret_cast<const void*>(&seg_pass_kernel<kSegThreads3, kSegItems3, true, 3>)},
      reinterpret_cast<const void*>(&local_sort_kernel<kTinyThreads, kLocalItems, false>),
      reinterpret_cast<const void*>(&local_sort_kernel<kTinyThreads, kLocalItems, true>),
      reinterpret_cast<const void*>(&local_sort_kernel<kSmallThreads, kLocalItems, false>),
      reinterpret_cast<const void*>(&local_sort_kernel<kSmallThreads, kLocalItems, true>),
      reinterpret_cast<const void*>(&seg_hist_kernel<kSegHistThreads, false>),
      reinterpret_cast<const void*>(&seg_hist_kernel<kSegHistThreads, true>),
      size_t(kMaxDigits) * 256 * 32 * 4,
  };
  return &k;
}

cudaError_t launch_seg_plan(const SegPlanArgs& a, cudaStream_t s) {
  seg_plan_kernel<<<1, 1024, 0, s>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_seg_hist(const SegHistArgs& a, unsigned grid, cudaStream_t s) {
  if (a.num_digits < 1 || a.num_digits > kMaxDigits) return cudaErrorInvalidValue;
  for (int j = 0; j < a.num_digits; ++j)  // the kernel counts the key's low bytes
    if (a.dig[j].shift != uint32_t(8 * j) || a.dig[j].width != 8u) return cudaErrorInvalidValue;
  const size_t smem = size_t(a.num_digits) * 256 * 32 * 4;
  if (is_identity(a.xform)) seg_hist_kernel<kSegHistThreads, false><<<grid, kSegHistThreads, smem, s>>>(a);
  else seg_hist_kernel<kSegHistThreads, true><<<grid, kSegHistThreads, smem, s>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_seg_scan(const SegScanArgs& a, unsigned grid, cudaStream_t s) {
  seg_scan_kernel<<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_seg_pass(const SegPassArgs& a, bool pairs, int shape, unsigned grid, cudaStream_t s) {
  if (shape == 2)
    return pairs ? launch_seg_pass<kSegThreads3, kSegItems3, true, 3>(a, grid, s)
                 : launch_seg_pass<kSegThreads3, kSegItems3, false, 3>(a, grid, s);
  if (shape == 0)
    return pairs ? launch_seg_pass<kSegThreads, kSegItemsSmall, true, 2>(a, grid, s)
                 : launch_seg_pass<kSegThreads, kSegItemsSmall, false, 2>(a, grid, s);
  return pairs ? launch_seg_pass<kSegThreads, kSegItemsPairs, true, 2>(a, grid, s)
               : launch_seg_pass<kSegThreads, kSegItemsKeys, false, 2>(a, grid, s);
}
cudaError_t launch_local_sort(const LocalArgs& a, bool small, bool pairs, unsigned grid, cudaStream_t s) {
  if (small)
    return pairs ? launch_local<kSmallThreads, kLocalItems, true>(a, grid, s)
                 : launch_local<kSmallThreads, kLocalItems, false>(a, grid, s);
  return pairs ? launch_local<kTinyThreads, kLocalItems, true>(a, grid, s)
               : launch_local<kTinyThreads, kLocalItems, false>(a, grid, s);
}
cudaError_t launch_bases_to_offsets(const uint32_t* bases, uint32_t num, uint64_t n, uint64_t* seg_off,
                                    cudaStream_t s) {
  bases_to_offsets_kernel<<<(num + 256) / 256, 256, 0, s>>>(bases, num, n, seg_off);
  return cudaGetLastError();
}

}  // namespace rs
