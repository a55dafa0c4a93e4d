// One LSD distribution pass by a digit, in a single read and write of the
// keys ("onesweep"): per tile, a stable rank of every key by its digit, a
// chained scan across tiles for the per-(tile, digit) output offset, and a
// scatter staged through shared memory so that keys of one digit leave the
// tile as one contiguous run.
//
// Paper: the pass is the bucketing/distribution step of Sec. 3.2 (count per
// bucket, cumulative totals, the partial sort grouping keys by bucket in
// ascending order, distribution of contiguous bucket ranges), done exactly:
// the per-cell-per-bucket offsets the paper chose not to compute (which
// left up to 128 elements misplaced, fixed later by post-balancing) come
// here from the chained scan, so no repair phase is needed.  Stability is
// what makes the repeated low-to-high passes a sort (Sec. 3.3.1) and keeps
// the order inside a bucket across the distribution (Sec. 5).
//
// Per tile (TILE = THREADS * ITEMS keys, tiles handed out by an atomic
// ticket so that every predecessor of a tile is already running):
//  1. load: warp w takes keys [w*32*ITEMS, (w+1)*32*ITEMS) of the tile,
//     item j of lane l being key w*32*ITEMS + j*32 + l (coalesced);
//  2. rank: per item, lanes with the same digit find each other through a
//     per-warp shared-memory table of lane masks (atomicOr, read back); the
//     highest such lane bumps the warp's private 16-bit counter for the
//     digit by the group size; a lane's rank within its warp is the counter
//     before the bump plus the number of group lanes below it.
//     Warp-private counters keep the rank order equal to the input order
//     (stability);
//  3. per digit: the tile's count (sum over warps) is published at once
//     as an "aggregate" status word; the counters are rewritten as
//     exclusive (digit, warp) prefixes, giving each key its position in the
//     digit-sorted tile;
//  4. lookback: walk back over earlier tiles' status words, a window of
//     them per round, adding aggregates until an "inclusive" word, then
//     publish this tile's inclusive count; waits are bounded;
//  5. stage keys (and values) in shared memory at their tile positions
//     (the lookback may also run after this step: EARLY_LB = false);
//  6. write the staged keys out in tile order, each to base[digit] + (keys
//     of the digit in earlier tiles) + (position within the digit here).
#pragma once

#include <type_traits>

#include "rs_device.cuh"
#include "rs_internal.h"

namespace rs {

// Width of the per-warp lane-mask table: 2^kMaskBits slots indexed by the
// digit's low kMaskBits bits; wider digits tell their remaining bits apart
// with one ballot per bit.  (A 32-slot table, one slot per shared-memory
// bank, avoids the table's bank conflicts but its three extra ballots per
// 8-bit key cost more issue slots than the conflicts: measured 312 vs 283 us
// per 2^26-key pass on GB300.)
constexpr int kMaskBits = 8;
constexpr uint32_t kMaskSlots = 1u << kMaskBits;

// DPT consecutive 16-bit counters, two per 32-bit word.  Sums of two halves
// never carry into each other because every count is at most TILE < 2^16.
template <int DPT>
struct CntVec {
  static constexpr int W = (DPT + 1) / 2;
  uint32_t w[W];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < W; ++i) w[i] = 0;
  }
  __device__ __forceinline__ void add(const CntVec& o) {
#pragma unroll
    for (int i = 0; i < W; ++i) w[i] += o.w[i];
  }
  __device__ __forceinline__ uint32_t half(int k) const { return (w[k >> 1] >> (16 * (k & 1))) & 0xffffu; }
  __device__ __forceinline__ void set_half(int k, uint32_t v) {
    w[k >> 1] = (w[k >> 1] & ~(0xffffu << (16 * (k & 1)))) | (v << (16 * (k & 1)));
  }
  __device__ __forceinline__ void load(const uint16_t* p) {
    if constexpr (DPT == 1) {
      w[0] = *p;
    } else if constexpr (DPT == 2) {
      w[0] = *reinterpret_cast<const uint32_t*>(p);
    } else if constexpr (DPT == 4) {
      const uint2 v = *reinterpret_cast<const uint2*>(p);
      w[0] = v.x;
      w[1] = v.y;
    } else {
      static_assert(DPT == 8, "digits per thread must be 1, 2, 4 or 8");
      const uint4 v = *reinterpret_cast<const uint4*>(p);
      w[0] = v.x;
      w[1] = v.y;
      w[2] = v.z;
      w[3] = v.w;
    }
  }
  __device__ __forceinline__ void store(uint16_t* p) const {
    if constexpr (DPT == 1) {
      *p = uint16_t(w[0]);
    } else if constexpr (DPT == 2) {
      *reinterpret_cast<uint32_t*>(p) = w[0];
    } else if constexpr (DPT == 4) {
      *reinterpret_cast<uint2*>(p) = make_uint2(w[0], w[1]);
    } else {
      *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
};

// NV: payload words moved with every key (0 = keys only, 1 = key + value,
// 2 = key + two words, e.g. the other half of a 64-bit key and a value).
template <int R, int THREADS, int ITEMS, int NV>
struct OnesweepLayout {
  static constexpr int DIGITS = 1 << R;
  static constexpr int WARPS = THREADS / 32;
  static constexpr int TILE = THREADS * ITEMS;
  // threads doing the per-digit work, and digits per such thread
  static constexpr int DTH = DIGITS < THREADS ? DIGITS : THREADS;
  static constexpr int DPT = DIGITS / DTH;
  // per-warp lane-mask table on the digit's low 8 bits, then per-warp
  // 16-bit running counters per digit
  static constexpr size_t MASK_BYTES = size_t(WARPS) * kMaskSlots * 4;
  static constexpr size_t CNT_BYTES = size_t(WARPS) * DIGITS * 2;
  static constexpr size_t RANK_BYTES = MASK_BYTES + CNT_BYTES;
  static constexpr size_t BUF_BYTES = size_t(TILE) * 4 * (1 + NV);
  static constexpr size_t UNION_BYTES = ((RANK_BYTES > BUF_BYTES ? RANK_BYTES : BUF_BYTES) + 15) / 16 * 16;
  static constexpr size_t OFF_GOFF = UNION_BYTES;
  static constexpr size_t OFF_WARP = OFF_GOFF + size_t(DIGITS) * 4;
  static constexpr size_t OFF_TILE = OFF_WARP + 32 * 4;
  static constexpr size_t SMEM = OFF_TILE + 16;
  static_assert(THREADS % 32 == 0 && THREADS <= 1024, "block shape");
  static_assert(TILE < 65536, "ranks are 16-bit");
  static_assert(DIGITS % DTH == 0, "digits must split evenly over threads");
  static_assert(RANK_BYTES % 16 == 0, "rank tables are cleared in 16-byte units");
  static_assert(R >= 8 && R <= 13, "digits of 8 to 13 bits");
};

// Vector relaxed load of 4 consecutive 32-bit status words (each word is
// read single-copy atomically; the four need not be read together).
__device__ __forceinline__ uint4 ld_relaxed4(const uint32_t* p) {
  uint4 v;
  asm volatile("ld.relaxed.gpu.global.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p)
               : "memory");
  return v;
}

// Exclusive prefix, over the earlier tiles of the same segment (tiles
// first .. tile-1), of the counts of this thread's DPT digits d0 ..
// d0+DPT-1 (decoupled lookback).  Reads a window of LB predecessors per round
// (LB * DPT loads in flight per thread).  Waits on a predecessor that has not
// published are bounded (kSpinLimit rounds), after which the error word is
// raised.
template <int DIGITS, int DPT, typename S, int LB>
__device__ __forceinline__ void lookback(const S* st, uint32_t tile, uint32_t first, int d0, uint32_t parity,
                                         uint32_t* err, uint32_t (&prefix)[DPT]) {
#pragma unroll
  for (int k = 0; k < DPT; ++k) prefix[k] = 0;
  if (tile == first) return;
  const int lo = int(first);
  constexpr bool VEC = (sizeof(S) == 4) && (DPT % 4 == 0);
  uint32_t spins = 0;
  if constexpr (VEC) {
    // one cursor for all DPT digits: rows are published whole, so the
    // digits of a thread move back together
    constexpr int NV = DPT / 4;
    int nr[DPT];  // next row each digit still has to add
#pragma unroll
    for (int k = 0; k < DPT; ++k) nr[k] = int(tile) - 1;
    uint32_t pending = (DPT >= 32) ? 0xffffffffu : ((1u << DPT) - 1u);
    while (pending) {
      int c = lo - 1;
#pragma unroll
      for (int k = 0; k < DPT; ++k)
        if (pending & (1u << k)) c = nr[k] > c ? nr[k] : c;
      uint4 w[LB][NV];
#pragma unroll
      for (int i = 0; i < LB; ++i)
#pragma unroll
        for (int v = 0; v < NV; ++v)
          if (c - i >= lo)
            w[i][v] = ld_relaxed4(reinterpret_cast<const uint32_t*>(st) + size_t(c - i) * DIGITS + d0 + 4 * v);
      bool stalled = false;
#pragma unroll
      for (int k = 0; k < DPT; ++k) {
#pragma unroll
        for (int i = 0; i < LB; ++i) {
          if (!(pending & (1u << k)) || nr[k] != c - i) continue;  // not this digit's next row
          if (c - i < lo) break;
          const uint4 q = w[i][k / 4];
          const uint32_t x = (k & 3) == 0 ? q.x : (k & 3) == 1 ? q.y : (k & 3) == 2 ? q.z : q.w;
          if (!status_ready<S>(S(x), parity)) {
            stalled = true;
            continue;
          }
          prefix[k] += status_count<S>(S(x));
          if (status_inclusive<S>(S(x))) pending &= ~(1u << k);
          else --nr[k];
        }
        if ((pending & (1u << k)) && nr[k] < lo) {  // cannot happen: the first tile is inclusive
          pending &= ~(1u << k);
          atomicOr(err, kErrTimeout);
        }
      }
      if (pending && stalled) {
        if (++spins > kSpinLimit) {
          atomicOr(err, kErrTimeout);
          return;
        }
        if (spins > 16) __nanosleep(100);
      }
    }
  } else {
    int pred[DPT];
#pragma unroll
    for (int k = 0; k < DPT; ++k) pred[k] = int(tile) - 1;
    uint32_t pending = (1u << DPT) - 1u;
    while (pending) {
      S w[DPT][LB];
#pragma unroll
      for (int k = 0; k < DPT; ++k)
#pragma unroll
        for (int i = 0; i < LB; ++i)
          if ((pending & (1u << k)) && pred[k] - i >= lo) w[k][i] = ld_relaxed(st + size_t(pred[k] - i) * DIGITS + d0 + k);
      bool stalled = false;
#pragma unroll
      for (int k = 0; k < DPT; ++k) {
        if (!(pending & (1u << k))) continue;
#pragma unroll
        for (int i = 0; i < LB; ++i) {
          if (!(pending & (1u << k))) break;
          if (pred[k] < lo) {  // cannot happen: the first tile is inclusive
            pending &= ~(1u << k);
            atomicOr(err, kErrTimeout);
            break;
          }
          const S x = w[k][i];
          if (!status_ready<S>(x, parity)) {
            stalled = true;
            break;
          }
          prefix[k] += status_count<S>(x);
          if (status_inclusive<S>(x)) pending &= ~(1u << k);
          else --pred[k];
        }
      }
      if (pending && stalled) {
        if (++spins > kSpinLimit) {
          atomicOr(err, kErrTimeout);
          return;
        }
        if (spins > 16) __nanosleep(100);
      }
    }
  }
}

// Stable rank of ITEMS keys per thread within their warp (item j of lane l
// is the warp's key j*32 + l).  Lanes holding the same digit find each other
// through the warp's table of lane masks (shared-memory atomicOr, then a
// read-back) indexed by the digit's low kMaskBits bits; the other bits are
// split off with one ballot per bit.  The highest lane of a
// group advances the warp's running count for the digit and clears the
// table slot.  A warp whose 32 digits are all equal skips the table.  Ranks
// are < 2^16, two per register.  wm / wc: this warp's mask table
// (kMaskSlots words, zero) and counters (2^R halfwords, zero on the first
// call).
template <int R, int ITEMS>
__device__ __forceinline__ void warp_rank(const uint32_t (&key)[ITEMS], uint32_t shift, uint32_t width, uint32_t* wm,
                                          uint16_t* wc, uint32_t (&rk)[(ITEMS + 1) / 2]) {
  static_assert(R <= 16, "two digits share the uniformity test word");
  const int lane = threadIdx.x & 31;
  const uint32_t lt = lanemask_lt(), gt = lanemask_gt();
  auto rank_one = [&](int j, uint32_t d, bool uniform) {
    uint32_t r;
    if (uniform) {
      const uint32_t before = wc[d];
      __syncwarp();
      if (lane == 31) wc[d] = uint16_t(before + 32u);
      __syncwarp();
      r = before + lane;
    } else {
      // digits of at most kMaskBits bits index the table directly
      const uint32_t lo = R <= kMaskBits ? d : (d & (kMaskSlots - 1u));
      uint32_t same_hi = 0xffffffffu;
#pragma unroll
      for (int b = kMaskBits; b < R; ++b) {
        const uint32_t bit = (d >> b) & 1u;
        const uint32_t bl = __ballot_sync(0xffffffffu, bit);
        same_hi &= bit ? bl : ~bl;
      }
      atomicOr(&wm[lo], 1u << lane);
      __syncwarp();
      const uint32_t slot = wm[lo];
      const uint32_t peers = slot & same_hi;
      const uint32_t before = wc[d];
      __syncwarp();
      if ((peers & gt) == 0) wc[d] = uint16_t(before + __popc(peers));
      if ((slot & gt) == 0) wm[lo] = 0u;
      __syncwarp();
      r = before + __popc(peers & lt);
    }
    if (j & 1) rk[j >> 1] |= r << 16;
    else rk[j >> 1] = r;
  };
  // Items two at a time: one shuffle and one vote tell whether both digits
  // are the same in every lane (then the counters move by 32 without the
  // mask table); otherwise both take the table, which is right either way.
#pragma unroll
  for (int j = 0; j < ITEMS; j += 2) {
    const uint32_t d0 = digit_of(key[j], shift, width);
    const uint32_t d1 = j + 1 < ITEMS ? digit_of(key[j + 1], shift, width) : d0;
    const uint32_t pk = d0 | (d1 << 16);
    const bool uniform = __all_sync(0xffffffffu, pk == __shfl_sync(0xffffffffu, pk, 0));
    rank_one(j, d0, uniform);
    if (j + 1 < ITEMS) rank_one(j + 1, d1, uniform);
  }
}

// Where one tile's keys come from and go to.
struct TileJob {
  uint32_t tile;          // row of the tile in the status array
  uint32_t first;         // first tile of the tile's segment (the lookback stops there)
  size_t base;            // index of the tile's first key in the source array
  uint32_t valid;         // keys in the tile (<= TILE)
  uint32_t out_start;     // output index of the segment's first key
  uint32_t out_end;       // output indexes must stay below this
  const uint32_t* bases;  // [2^R]: the segment's keys with a smaller digit
};

// One tile of an LSD pass (steps 1-6 above).  The rank tables must be zero
// on entry (the caller clears them and synchronises the block).
// Interleaved two-word elements of the first and the last executed pass (in
// and out are null on the other passes): 64-bit keys, whose word `high` is
// this pass's key and whose other word rides as payload word 1, or 64-bit
// values, payload words 1 and 2.
// With iota, the first executed pass makes the last payload word the
// element's index in the input; with gout, the last executed pass writes
// gather[that index] to gout in its place (values sorted by an index that
// the passes carry instead of the values themselves; kernels with two
// payload words and 64-bit keys).
struct PairIO {
  const uint2* in;
  uint2* out;
  int key;        // 1: 64-bit keys; 0: 64-bit values
  uint32_t high;  // 64-bit keys: this pass's digit lies in the high word
  KeyXform64 x;   // 64-bit keys: their order map
  int iota;
  const uint2* gather;
  uint2* gout;
  uint32_t n;     // bound of a gathered index
};

// PIO: the PairIO paths are compiled in (kernels of the 64-bit sorts); the
// plain kernels carry none of that code.
template <int R, int THREADS, int ITEMS, int NV, typename S, bool EARLY_LB, bool PIO = false>
__device__ __forceinline__ void onesweep_tile(const TileJob& job, const uint32_t* kin, uint32_t* kout,
                                              const uint32_t* vin, uint32_t* vout, const uint32_t* vin2,
                                              uint32_t* vout2, const PairIO& pio, uint32_t shift, uint32_t width,
                                              S* status, uint32_t parity, uint32_t* err, KeyXform xin, KeyXform xout,
                                              unsigned char* smem) {
  using L = OnesweepLayout<R, THREADS, ITEMS, NV>;
  constexpr int DIGITS = L::DIGITS, WARPS = L::WARPS, TILE = L::TILE;
  constexpr int DTH = L::DTH, DPT = L::DPT;
  // rank tables ([WARPS][kMaskSlots] lane masks, then [WARPS][DIGITS] 16-bit
  // counters), aliased by the staging buffer once positions are final
  uint32_t* s_mask = reinterpret_cast<uint32_t*>(smem);
  uint16_t* s_cnt = reinterpret_cast<uint16_t*>(smem + L::MASK_BYTES);
  uint32_t* s_buf = reinterpret_cast<uint32_t*>(smem);
  uint32_t* s_goff = reinterpret_cast<uint32_t*>(smem + L::OFF_GOFF);
  uint32_t* s_warp = reinterpret_cast<uint32_t*>(smem + L::OFF_WARP);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t tile = job.tile, valid = job.valid;

  // 1p. the payload words of a full tile that step 5 reads from planes,
  // prefetched into L2 (not those read interleaved or made from the index)
  if constexpr (NV >= 1) {
    if (valid == TILE && !(PIO && pio.in)) {
      if ((reinterpret_cast<uintptr_t>(vin + job.base) & 15u) == 0) prefetch_l2_tile(vin + job.base, uint32_t(TILE) * 4u);
      if constexpr (NV >= 2) {
        if (vin2 && !(PIO && pio.iota) && (reinterpret_cast<uintptr_t>(vin2 + job.base) & 15u) == 0)
          prefetch_l2_tile(vin2 + job.base, uint32_t(TILE) * 4u);
      }
    }
  }

  // 1. load the keys
  uint32_t key[ITEMS];
  const size_t wbase = job.base + size_t(warp) * 32 * ITEMS + lane;
  const size_t wend = job.base + valid;
  // 64-bit keys read interleaved keep the other word of their order map in
  // the first payload section of the staging buffer, at the key's place in
  // the tile, while the rank tables are in use (they fit below it); where
  // they do not fit, the payload stage reads the word again (from L2).
  constexpr bool STASH = L::RANK_BYTES <= size_t(TILE) * 4;
  const uint32_t stash = TILE + warp * 32 * ITEMS + lane;
  if (PIO && NV >= 1 && pio.key && pio.in) {
    uint2 m[ITEMS];  // every load in flight before the first use
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      const size_t idx = wbase + j * 32;
      m[j] = (valid == TILE || idx < wend) ? ld_stream2(pio.in + idx) : make_uint2(0xffffffffu, 0xffffffffu);
    }
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      // past the end: the largest key (its map is never taken)
      const size_t idx = wbase + j * 32;
      if (valid == TILE || idx < wend) m[j] = map64(m[j], pio.x);
      key[j] = pio.high ? m[j].y : m[j].x;
      if constexpr (STASH) s_buf[stash + j * 32] = pio.high ? m[j].x : m[j].y;
    }
  } else if (valid == TILE) {
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) key[j] = ld_stream(kin + wbase + j * 32);
    if (!is_identity(xin)) {
#pragma unroll
      for (int j = 0; j < ITEMS; ++j) key[j] = to_ordered(key[j], xin);
    }
  } else {
    // Keys past the end act as 0xFFFFFFFF: their digit is the largest and
    // they come after every real key, so they sort to the tile's tail and
    // are never written.
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      const size_t idx = wbase + j * 32;
      key[j] = idx < wend ? to_ordered(kin[idx], xin) : 0xffffffffu;
    }
  }

  // 2. rank within the warp
  uint32_t rk[(ITEMS + 1) / 2];
  warp_rank<R, ITEMS>(key, shift, width, s_mask + warp * kMaskSlots, s_cnt + warp * DIGITS, rk);
  __syncthreads();

  // 3. per-digit tile counts -> aggregate status; counts -> exclusive
  // (digit, warp) prefixes, i.e. where each warp's run of a digit starts
  const int d0 = tid * DPT;
  uint32_t tot[DPT], loff[DPT];
  uint32_t my_sum = 0;
  if (tid < DTH) {
    CntVec<DPT> run;
    run.zero();
#pragma unroll 4
    for (int wi = 0; wi < WARPS; ++wi) {
      CntVec<DPT> v;
      v.load(s_cnt + wi * DIGITS + d0);
      run.add(v);
    }
    S* mine = status + size_t(tile) * DIGITS + d0;
#pragma unroll
    for (int k = 0; k < DPT; ++k) {
      tot[k] = run.half(k);
      my_sum += tot[k];
      st_relaxed(mine + k, status_word<S>(parity, tile == job.first, tot[k]));
    }
  }
  const uint32_t excl = block_exclusive_sum<THREADS>(my_sum, s_warp);
  if (tid < DTH) {
    uint32_t r = excl;
#pragma unroll
    for (int k = 0; k < DPT; ++k) {
      loff[k] = r;
      r += tot[k];
    }
    CntVec<DPT> run;
    run.zero();
#pragma unroll
    for (int k = 0; k < DPT; ++k) run.set_half(k, loff[k]);
#pragma unroll 4
    for (int wi = 0; wi < WARPS; ++wi) {
      CntVec<DPT> v;
      v.load(s_cnt + wi * DIGITS + d0);
      run.store(s_cnt + wi * DIGITS + d0);
      run.add(v);
    }
  }

  // 4. chained scan over the segment's earlier tiles (decoupled lookback),
  // either now or after the tile is staged
  auto do_lookback = [&]() {
    if (tid < DTH) {
      uint32_t prefix[DPT];
      // About eight status words per thread and round: the nearest
      // inclusive predecessor is usually a few tiles back, and wider windows
      // cost more issue slots than the rounds they save (GB300, 2^26 keys:
      // 271 vs 282 us per 512 x 24 pass with 8 vs 32 words, 390 vs 434 us
      // per 11-bit pass with 4 vs 16 rows of two digits).
      constexpr int LBW = (8 / DPT) > 1 ? 8 / DPT : 1;
      lookback<DIGITS, DPT, S, LBW>(status, tile, job.first, d0, parity, err, prefix);
      if (tile != job.first) {
        S* mine = status + size_t(tile) * DIGITS + d0;
#pragma unroll
        for (int k = 0; k < DPT; ++k) st_relaxed(mine + k, status_word<S>(parity, true, prefix[k] + tot[k]));
      }
#pragma unroll
      for (int k = 0; k < DPT; ++k) s_goff[d0 + k] = job.out_start + job.bases[d0 + k] + prefix[k] - loff[k];
    }
  };
  if constexpr (EARLY_LB) do_lookback();
  __syncthreads();

  // 5. tile positions; stage the tile in shared memory in digit order
#pragma unroll
  for (int j = 0; j < ITEMS; ++j) {
    const uint32_t pos = s_cnt[warp * DIGITS + digit_of(key[j], shift, width)];
    if (j & 1) rk[j >> 1] += pos << 16;
    else rk[j >> 1] += pos;
  }
  __syncthreads();  // rank tables are dead; the staging buffer reuses them
#pragma unroll
  for (int j = 0; j < ITEMS; ++j) s_buf[(rk[j >> 1] >> (16 * (j & 1))) & 0xffffu] = key[j];
  // payload words, one at a time (each staged in its own TILE-word section)
  bool staged = false;
  if constexpr (PIO && NV >= 2) {
    if (pio.in && !pio.key) {  // 64-bit values read interleaved: words 1 and 2, half a row at a time
      constexpr int H = (ITEMS + 1) / 2;
#pragma unroll
      for (int h = 0; h < ITEMS; h += H) {
        uint2 v2[H];
#pragma unroll
        for (int j = 0; j < H; ++j) {
          const size_t idx = wbase + (h + j) * 32;
          v2[j] = (h + j < ITEMS && (valid == TILE || idx < wend)) ? ld_stream2(pio.in + idx) : make_uint2(0u, 0u);
        }
#pragma unroll
        for (int j = 0; j < H; ++j) {
          if (h + j < ITEMS) {
            const uint32_t pos = (rk[(h + j) >> 1] >> (16 * ((h + j) & 1))) & 0xffffu;
            s_buf[TILE + pos] = v2[j].x;
            s_buf[2 * TILE + pos] = v2[j].y;
          }
        }
      }
      staged = true;
    }
  }
  if (!staged) {
#pragma unroll
    for (int w = 0; w < NV; ++w) {
      const uint32_t* src = w == 0 ? vin : vin2;
      uint32_t val[ITEMS];
      if (PIO && NV >= 2 && w == NV - 1 && pio.iota) {  // the element's index in the input
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) val[j] = uint32_t(wbase + j * 32);
      } else if (PIO && w == 0 && pio.key && pio.in) {  // the other word of an interleaved 64-bit key
        if constexpr (STASH) {
#pragma unroll
          for (int j = 0; j < ITEMS; ++j) val[j] = s_buf[stash + j * 32];
          __syncthreads();  // every stashed word is read before the section is overwritten
        } else {
#pragma unroll
          for (int j = 0; j < ITEMS; ++j) {
            const size_t idx = wbase + j * 32;
            uint2 m = make_uint2(0u, 0u);
            if (valid == TILE || idx < wend) m = map64(ld_stream2(pio.in + idx), pio.x);
            val[j] = pio.high ? m.x : m.y;
          }
        }
      } else if (valid == TILE) {
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) val[j] = ld_stream(src + wbase + j * 32);
      } else {
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
          const size_t idx = wbase + j * 32;
          val[j] = idx < wend ? src[idx] : 0u;
        }
      }
#pragma unroll
      for (int j = 0; j < ITEMS; ++j) s_buf[(1 + w) * TILE + ((rk[j >> 1] >> (16 * (j & 1))) & 0xffffu)] = val[j];
    }
  }
  if constexpr (!EARLY_LB) do_lookback();
  __syncthreads();

  // 6. write out in tile order: runs of one digit go to consecutive
  // addresses.  The range check only guards against a corrupted offset (it
  // raises an error bit instead of writing out of bounds).
  // Keys leave through the inverse of the order map when this pass writes
  // the final order (the loop is written twice so that the identity case
  // pays nothing).
  // The last pass of an interleaved sort writes the two words of each
  // element as one 8-byte store (PAIR 1: a 64-bit key, through the inverse of
  // its order map; PAIR 2: a 64-bit value).
  // GATHER (64-bit keys): the second payload word is an input index, and
  // gather[index] goes out in its place (an index out of range is skipped
  // and reported).  These are random reads; issuing several before their
  // stores measured no faster.
  bool oob = false;
  const uint32_t span = job.out_end - job.out_start;
  auto gather_put = [&](uint32_t g, uint32_t ix) {
    if (ix < pio.n) pio.gout[g] = ld_stream2(pio.gather + ix);
    else oob = true;
  };
  auto write_out = [&](auto invert, auto pair, auto gather) {
    constexpr int PAIR = decltype(pair)::value;
    constexpr bool GATHER = decltype(gather)::value;
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
      const uint32_t i = k * THREADS + tid;
      if (valid == TILE || i < valid) {
        const uint32_t kk = s_buf[i];
        const uint32_t g = s_goff[digit_of(kk, shift, width)] + i;
        if (g - job.out_start < span) {  // out_start <= g < out_end
          if constexpr (PAIR == 1) {
            const uint32_t o = s_buf[TILE + i];
            pio.out[g] = unmap64(pio.high ? make_uint2(o, kk) : make_uint2(kk, o), pio.x);
            if constexpr (NV >= 2) {
              if constexpr (GATHER) gather_put(g, s_buf[2 * TILE + i]);
              else vout2[g] = s_buf[2 * TILE + i];
            }
          } else {
            kout[g] = decltype(invert)::value ? from_ordered(kk, xout) : kk;
            if constexpr (PAIR == 2) {
              pio.out[g] = make_uint2(s_buf[TILE + i], s_buf[2 * TILE + i]);
            } else {
              if constexpr (NV >= 1) vout[g] = s_buf[TILE + i];
              if constexpr (NV >= 2) vout2[g] = s_buf[2 * TILE + i];
            }
          }
        } else {
          oob = true;
        }
      }
    }
  };
  using P0 = std::integral_constant<int, 0>;
  using NG = std::false_type;
  if constexpr (PIO && NV >= 1) {
    if (pio.out && pio.key) {
      if (NV >= 2 && pio.gout) write_out(std::false_type{}, std::integral_constant<int, 1>{}, std::true_type{});
      else write_out(std::false_type{}, std::integral_constant<int, 1>{}, NG{});
      if (oob) atomicOr(err, kErrBounds);
      return;
    }
  }
  if constexpr (PIO && NV >= 2) {
    if (pio.out) {
      if (is_identity(xout)) write_out(std::false_type{}, std::integral_constant<int, 2>{}, NG{});
      else write_out(std::true_type{}, std::integral_constant<int, 2>{}, NG{});
      if (oob) atomicOr(err, kErrBounds);
      return;
    }
  }
  if (is_identity(xout)) write_out(std::false_type{}, P0{}, NG{});
  else write_out(std::true_type{}, P0{}, NG{});
  if (oob) atomicOr(err, kErrBounds);
}

// Clears the rank tables and takes the block's tile ticket.
template <int R, int THREADS, int ITEMS, int NV>
__device__ __forceinline__ uint32_t begin_tile(uint32_t* counter, unsigned char* smem) {
  using L = OnesweepLayout<R, THREADS, ITEMS, NV>;
  uint32_t* s_tile = reinterpret_cast<uint32_t*>(smem + L::OFF_TILE);
  uint4* c4 = reinterpret_cast<uint4*>(smem);
  for (int i = threadIdx.x; i < int(L::RANK_BYTES / 16); i += THREADS) c4[i] = make_uint4(0u, 0u, 0u, 0u);
  if (threadIdx.x == 0) *s_tile = atomicAdd(counter, 1u);
  __syncthreads();
  return *s_tile;
}

// The plain pass: tile i covers keys [i * TILE, (i + 1) * TILE) of one array.
template <int R, int THREADS, int ITEMS, int NV, typename S, int MINB, bool EARLY_LB, bool PIO>
__global__ void __launch_bounds__(THREADS, MINB) onesweep_kernel(const PassArgs a) {
  using L = OnesweepLayout<R, THREADS, ITEMS, NV>;
  extern __shared__ __align__(16) unsigned char smem[];
  const Route route = route_of(a.skip, a.pass, a.num_passes);
  if (!route.active) return;
  const uint32_t* kin = route.src == BUF_IN ? a.keys_in : (route.src == BUF_OUT ? a.keys_out : a.keys_alt);
  uint32_t* kout = route.dst == BUF_OUT ? a.keys_out : a.keys_alt;
  const uint32_t *vin = nullptr, *vin2 = nullptr;
  uint32_t *vout = nullptr, *vout2 = nullptr;
  if constexpr (NV >= 1) {
    vin = route.src == BUF_IN ? a.vals_in : (route.src == BUF_OUT ? a.vals_out : a.vals_alt);
    vout = route.dst == BUF_OUT ? a.vals_out : a.vals_alt;
  }
  if constexpr (NV >= 2) {
    vin2 = route.src == BUF_IN ? a.vals2_in : (route.src == BUF_OUT ? a.vals2_out : a.vals2_alt);
    vout2 = route.dst == BUF_OUT ? a.vals2_out : a.vals2_alt;
  }
  PairIO pio{nullptr, nullptr, a.pair_key, a.key_high, a.x64, 0, a.gather, nullptr, a.n};
  if constexpr (PIO && NV >= 1) {
    if (route.src == BUF_IN) {
      pio.in = a.pair_in;
      pio.iota = a.iota;
    }
    if (route.last) {
      pio.out = a.pair_out;
      pio.gout = a.gather_out;
    }
  }
  const uint32_t tile = begin_tile<R, THREADS, ITEMS, NV>(a.tile_counter, smem);
  TileJob job;
  job.tile = tile;
  job.first = 0;
  job.base = size_t(tile) * L::TILE;
  const size_t left = size_t(a.n) - job.base;
  job.valid = left < size_t(L::TILE) ? uint32_t(left) : uint32_t(L::TILE);
  job.out_start = 0;
  job.out_end = a.n;
  job.bases = a.bases;
  onesweep_tile<R, THREADS, ITEMS, NV, S, EARLY_LB, PIO>(job, kin, kout, vin, vout, vin2, vout2, pio, a.shift,
                                                             a.width,
                                                        reinterpret_cast<S*>(a.status), route.parity, a.err,
                                                        route.src == BUF_IN ? a.xin : KeyXform{0u, 0u},
                                                        route.last ? a.xout : KeyXform{0u, 0u}, smem);
}

template <int R, int THREADS, int ITEMS, int NV, typename S, int MINB, bool EARLY_LB, bool PIO>
cudaError_t launch_onesweep(const PassArgs& a, unsigned grid, cudaStream_t s) {
  using L = OnesweepLayout<R, THREADS, ITEMS, NV>;
  onesweep_kernel<R, THREADS, ITEMS, NV, S, MINB, EARLY_LB, PIO><<<grid, THREADS, L::SMEM, s>>>(a);
  return cudaGetLastError();
}

template <int R, int THREADS, int ITEMS, int NV, typename S, int MINB, bool EARLY_LB, bool PIO = false>
OnesweepKernel make_onesweep(int shape_id) {
  using L = OnesweepLayout<R, THREADS, ITEMS, NV>;
  return OnesweepKernel{R,
                        shape_id,
                        THREADS,
                        ITEMS,
                        L::TILE,
                        NV >= 1,
                        sizeof(S) == 8,
                        L::SMEM,
                        &launch_onesweep<R, THREADS, ITEMS, NV, S, MINB, EARLY_LB, PIO>,
                        reinterpret_cast<const void*>(&onesweep_kernel<R, THREADS, ITEMS, NV, S, MINB, EARLY_LB, PIO>),
                        0,
                        NV,
                        PIO};
}

}  // namespace rs
