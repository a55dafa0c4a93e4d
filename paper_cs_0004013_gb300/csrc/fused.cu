// A whole sort of up to a few million keys in one launch.
//
// Paper: the same radix distribution as the pipeline of separate launches
// (the count loop and cumulative totals of Sec. 3.2, then one stable
// distribution per digit from the low one up, Sec. 3.3.1); only the launch
// structure differs.  For small inputs the pipeline's seven launches (clear,
// histogram, scans, four passes) cost more than the work, so here every tile
// of the array has its own block, all blocks are resident at once (a
// cooperative launch refuses otherwise), and the phases are separated by
// grid-wide barriers instead of launches:
//   1. each block counts the four byte digits of its tile and adds them into
//      the global histograms;                                    barrier
//   2. every block scans the histograms itself (they are small): digit bases
//      and the skip flags (a digit with one bucket holding every key);
//   3. for each executed digit: the block's tile goes through the pass of the
//      half-warp-group kernel (onesweep2.cuh), the lookback ordering the
//      tiles inside the pass;                                     barrier
// Loads use the L2 path (ld.global.cg): later passes read what other blocks
// wrote earlier in the same launch.  Every barrier wait is bounded: a block
// that waits too long raises the device error word and goes on, so the
// launch always ends.
#include <cstdint>

#include "onesweep2.cuh"

namespace rs {
namespace {

constexpr int kFusedThreads = 384;
// Tile shapes (index = fused shape): 384 x 24, 384 x 18 and 384 x 12.  A
// pass of the single launch lasts about one tile's chain of loads, ranking,
// lookback and write-out, so smaller tiles are faster while every tile still
// has an SM of its own (GB300: 2^19 keys in 39.5 us with 384 x 12 against
// 43.8 with 384 x 24) and slower once tiles share SMs (2^20 keys: 50.1
// against 47.4).
constexpr int kFusedItems[kFusedShapes] = {24, 18, 12};
constexpr int fused_min_blocks(int items) { return items <= 12 ? 3 : 2; }
// Status rows a digit thread reads per lookback round (GB300, 2^20 keys in
// 152 tiles of 384 x 18: the kernel takes 44.7 us with 8 rows per round,
// 47.8 with 16 and 62.1 with 32).
constexpr int kFusedLookback = 8;
// Rounds of a barrier wait (about 64 ns each) before it gives up.
constexpr uint32_t kBarrierSpinLimit = 1u << 21;

template <int NV, int ITEMS>
struct FusedLayout {
  using L = Onesweep2Layout<kFusedThreads, ITEMS, NV>;
  static constexpr size_t OFF_BASES = (L::SMEM + 15) / 16 * 16;  // [4][256]
  static constexpr size_t OFF_FLAGS = OFF_BASES + 4 * 256 * 4;   // [4] skip flags
  static constexpr size_t SMEM = OFF_FLAGS + 16;
};

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Arrival number `target` of the launch's monotone barrier counter.
__device__ __forceinline__ void grid_barrier(uint32_t* bar, uint32_t target, uint32_t* err) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(bar, 1u);
    uint32_t spins = 0;
    while (ld_acquire(bar) < target) {
      if (++spins > kBarrierSpinLimit) {
        atomicOr(err, kErrTimeout);
        break;
      }
      __nanosleep(32);
    }
    __threadfence();
  }
  __syncthreads();
}

template <int NV, int ITEMS>
__global__ void __launch_bounds__(kFusedThreads, fused_min_blocks(ITEMS)) fused_sort_kernel(const FusedArgs a) {
  using FL = FusedLayout<NV, ITEMS>;
  using L = typename FL::L;
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* s_bases = reinterpret_cast<uint32_t*>(smem + FL::OFF_BASES);
  uint32_t* s_flags = reinterpret_cast<uint32_t*>(smem + FL::OFF_FLAGS);
  uint32_t* s_cnt = reinterpret_cast<uint32_t*>(smem + L::OFF_TBL);  // [4][256] while counting
  const int tid = threadIdx.x;
  const uint32_t tile = blockIdx.x, tiles = gridDim.x;
  const uint32_t n = a.n;

  // 1. counts of the tile's four digits (order-mapped keys)
  for (int i = tid; i < 1024; i += kFusedThreads) s_cnt[i] = 0u;
  __syncthreads();
  {
    const uint32_t cnt = smem_addr(s_cnt);
    const uint64_t lo = uint64_t(tile) * L::TILE;
    const uint64_t hi = lo + L::TILE < n ? lo + L::TILE : n;
    for (uint64_t i = lo + tid; i < hi; i += kFusedThreads) {
      const uint32_t k = to_ordered(a.keys_in[i], a.xf);
#pragma unroll
      for (uint32_t j = 0; j < 4; ++j) sh_red_add(cnt + 4u * (256u * j + byte_digit(k, 0x4440u | j)), 1u);
    }
  }
  __syncthreads();
  for (int i = tid; i < 1024; i += kFusedThreads)
    if (s_cnt[i]) atomicAdd(a.hist + i, s_cnt[i]);
  grid_barrier(a.bar, tiles, a.err);

  // 2. bases and skip flags of every digit (each block for itself)
  if (tid < 4) s_flags[tid] = 0u;
  __syncthreads();
  for (int j = 0; j < 4; ++j) {
    if (tid < 256) {
      const uint32_t v = ld_pass<true>(a.hist + 256 * j + tid);
      if (v == n) s_flags[j] = 1u;  // one bucket holds every key: the digit moves nothing
      s_bases[256 * j + tid] = scan256_exclusive(v, reinterpret_cast<uint32_t*>(smem + L::OFF_SCAN));
    }
    __syncthreads();
  }

  // 3. the executed passes: the skipped digits are left out; if every digit
  // is skipped the last one still runs (a stable copy into keys_out).  The
  // executed passes alternate between keys_out and the alternate buffer so
  // that the last one lands in keys_out.
  uint32_t order = 0;  // the executed digits, one per byte, lowest first
  int m = 0;
  for (int j = 0; j < 4; ++j)
    if (!s_flags[j]) order |= uint32_t(j) << (8 * m++);
  if (m == 0) {
    order = 3u;
    m = 1;
  }
  for (int e = 0; e < m; ++e) {
    const int j = int((order >> (8 * e)) & 0xffu);
    uint4* t4 = reinterpret_cast<uint4*>(smem + L::OFF_TBL);
    for (int i = tid; i < int(L::TBL / 16); i += kFusedThreads) t4[i] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    const bool to_out = ((m - 1 - e) % 2) == 0;
    const bool from_out = e > 0 && ((m - e) % 2) == 0;
    Tile2Job job;
    job.tile = tile;
    job.n = n;
    job.kin = e == 0 ? a.keys_in : (from_out ? a.keys_out : a.keys_alt);
    job.kout = to_out ? a.keys_out : a.keys_alt;
    job.vin = nullptr;
    job.vout = nullptr;
    if constexpr (NV >= 1) {
      job.vin = e == 0 ? a.vals_in : (from_out ? a.vals_out : a.vals_alt);
      job.vout = to_out ? a.vals_out : a.vals_alt;
    }
    job.xin = e == 0 ? a.xf : KeyXform{0u, 0u};
    job.xout = e == m - 1 ? a.xf : KeyXform{0u, 0u};
    job.parity = uint32_t(e & 1) ^ 1u;
    job.status = a.status;
    job.bases = s_bases + 256 * j;
    job.shift = uint32_t(8 * j);
    job.err = a.err;
    bool unstable = false;  // the first executed pass of keys on a full tile: equal digits leave in any order
    if constexpr (NV == 0) unstable = e == 0 && (size_t(tile) + 1) * L::TILE <= size_t(n);
    if (unstable)
      onesweep2_tile<kFusedThreads, ITEMS, NV, uint32_t, false, kFusedLookback, true, true>(job, smem);
    else
      onesweep2_tile<kFusedThreads, ITEMS, NV, uint32_t, false, kFusedLookback, true, false>(job, smem);
    if (e + 1 < m) grid_barrier(a.bar, tiles * uint32_t(2 + e), a.err);
  }
}

}  // namespace

uint32_t fused_tile_keys(int shape) { return uint32_t(kFusedThreads * kFusedItems[shape]); }

template <int SH>
struct FusedShape {
  static constexpr int ITEMS = kFusedItems[SH];
  static size_t smem(bool pairs) { return pairs ? FusedLayout<1, ITEMS>::SMEM : FusedLayout<0, ITEMS>::SMEM; }
  static const void* func(bool pairs) {
    return pairs ? reinterpret_cast<const void*>(&fused_sort_kernel<1, ITEMS>)
                 : reinterpret_cast<const void*>(&fused_sort_kernel<0, ITEMS>);
  }
};
static_assert(kFusedShapes == 3, "one FusedShape per entry of kFusedItems");

size_t fused_smem(bool pairs, int shape) {
  return shape == 0 ? FusedShape<0>::smem(pairs) : shape == 1 ? FusedShape<1>::smem(pairs) : FusedShape<2>::smem(pairs);
}
const void* fused_func(bool pairs, int shape) {
  return shape == 0 ? FusedShape<0>::func(pairs) : shape == 1 ? FusedShape<1>::func(pairs) : FusedShape<2>::func(pairs);
}

cudaError_t launch_fused(const FusedArgs& a, unsigned tiles, bool pairs, int shape, cudaStream_t s) {
  FusedArgs args = a;
  void* params[] = {&args};
  return cudaLaunchCooperativeKernel(fused_func(pairs, shape), dim3(tiles), dim3(kFusedThreads), params,
                                     fused_smem(pairs, shape), s);
}

}  // namespace rs
