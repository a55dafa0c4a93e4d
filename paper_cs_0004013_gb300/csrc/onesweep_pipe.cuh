// The onesweep pass as a persistent, software-pipelined kernel (8-bit
// digits).
//
// Same arithmetic as onesweep_tile (rank, per-digit counts and aggregate
// status, exclusive prefixes, lookback, stable scatter), but each block loops
// over tiles and overlaps the two latency-bound steps with useful work:
//
//   iteration i (tile t_i, keys already in registers):
//     rank t_i, publish its aggregate counts, stage it into buffer i % 2;
//     take the next ticket and issue the loads of that tile's keys;
//     issue the first window of t_i's lookback;
//     write out tile t_{i-1} from buffer (i-1) % 2       <- overlaps the loads
//     finish t_i's lookback, publish its inclusive counts, keep its offsets.
//
// Tile t_i's own write-out waits one iteration, which gives its lookback the
// whole write-out of t_{i-1} to complete; the key loads of t_{i+1} are in
// flight during the same time.  Successors never wait for t_i's inclusive
// word specifically (they can use its aggregate and walk further back), so
// deferring it cannot deadlock.
#pragma once

#include "onesweep.cuh"

namespace rs {

template <int R, int THREADS, int ITEMS, bool PAIRS>
struct PipeLayout {
  static constexpr int DIGITS = 1 << R;
  static constexpr int WARPS = THREADS / 32;
  static constexpr int TILE = THREADS * ITEMS;
  static constexpr size_t MASK_BYTES = size_t(WARPS) * kMaskSlots * 4;
  static constexpr size_t CNT_BYTES = size_t(WARPS) * DIGITS * 2;
  static constexpr size_t RANK_BYTES = (MASK_BYTES + CNT_BYTES + 15) / 16 * 16;
  static constexpr size_t BUF_BYTES = size_t(TILE) * 4 * (PAIRS ? 2 : 1);
  static constexpr size_t OFF_BUF0 = RANK_BYTES;
  static constexpr size_t OFF_BUF1 = OFF_BUF0 + BUF_BYTES;
  static constexpr size_t OFF_GOFF = OFF_BUF1 + BUF_BYTES;  // [2][DIGITS]
  static constexpr size_t OFF_WARP = OFF_GOFF + size_t(2) * DIGITS * 4;
  static constexpr size_t OFF_TILE = OFF_WARP + 32 * 4;
  static constexpr size_t SMEM = OFF_TILE + 16;
  static_assert(THREADS >= DIGITS, "one thread per digit");
  static_assert(TILE < 65536, "ranks are 16-bit");
  static_assert(SMEM <= 227 * 1024, "shared memory");
};

// Lookback of one digit in windows of LB predecessors: issue the loads of a
// window now, consume them later.
template <typename S, int LB>
struct DigitLookback {
  S w[LB];
  int next;        // next row to add
  int issued;      // row of w[0]
  uint32_t prefix;
  bool done;
  uint32_t spins;

  __device__ __forceinline__ void start(uint32_t tile, uint32_t first) {
    next = int(tile) - 1;
    prefix = 0;
    done = tile == first;
    spins = 0;
  }
  __device__ __forceinline__ void issue(const S* st, int digits, int d, int first) {
    issued = next;
#pragma unroll
    for (int i = 0; i < LB; ++i)
      if (next - i >= first) w[i] = ld_relaxed(st + size_t(next - i) * digits + d);
  }
  // Adds the window's words up to the first inclusive one; returns false if
  // a word was not ready (the next issue starts there).
  __device__ __forceinline__ bool consume(int first, uint32_t parity, uint32_t* err) {
#pragma unroll
    for (int i = 0; i < LB; ++i) {
      if (done) return true;
      if (issued - i < first) {  // cannot happen: the first tile is inclusive
        atomicOr(err, kErrTimeout);
        done = true;
        return true;
      }
      const S x = w[i];
      if (!status_ready<S>(x, parity)) return false;
      prefix += status_count<S>(x);
      if (status_inclusive<S>(x)) done = true;
      else next = issued - i - 1;
    }
    return true;
  }
};

template <int R, int THREADS, int ITEMS, bool PAIRS, typename S, int MINB>
__global__ void __launch_bounds__(THREADS, MINB) onesweep_pipe_kernel(const PassArgs a) {
  using L = PipeLayout<R, THREADS, ITEMS, PAIRS>;
  constexpr int DIGITS = L::DIGITS, WARPS = L::WARPS, TILE = L::TILE;
  constexpr int LB = 8;
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* s_mask = reinterpret_cast<uint32_t*>(smem);
  uint16_t* s_cnt = reinterpret_cast<uint16_t*>(smem + L::MASK_BYTES);
  uint32_t* s_goff = reinterpret_cast<uint32_t*>(smem + L::OFF_GOFF);
  uint32_t* s_warp = reinterpret_cast<uint32_t*>(smem + L::OFF_WARP);
  uint32_t* s_tile = reinterpret_cast<uint32_t*>(smem + L::OFF_TILE);
  auto s_buf = [&](int i) { return reinterpret_cast<uint32_t*>(smem + ((i & 1) ? L::OFF_BUF1 : L::OFF_BUF0)); };

  const Route route = route_of(a.skip, a.pass, a.num_passes);
  if (!route.active) return;
  const uint32_t* kin = route.src == BUF_IN ? a.keys_in : (route.src == BUF_OUT ? a.keys_out : a.keys_alt);
  uint32_t* kout = route.dst == BUF_OUT ? a.keys_out : a.keys_alt;
  const uint32_t* vin = nullptr;
  uint32_t* vout = nullptr;
  if constexpr (PAIRS) {
    vin = route.src == BUF_IN ? a.vals_in : (route.src == BUF_OUT ? a.vals_out : a.vals_alt);
    vout = route.dst == BUF_OUT ? a.vals_out : a.vals_alt;
  }
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t num_tiles = uint32_t((size_t(a.n) + TILE - 1) / TILE);
  S* status = reinterpret_cast<S*>(a.status);
  const uint32_t shift = a.shift, width = a.width, parity = route.parity;
  // order map of the keys read from the input / written as the final order
  const KeyXform xin = route.src == BUF_IN ? a.xin : KeyXform{0u, 0u};
  const KeyXform xout = route.last ? a.xout : KeyXform{0u, 0u};

  auto clear_tables = [&]() {
    uint4* c4 = reinterpret_cast<uint4*>(smem);
    for (int i = tid; i < int(L::RANK_BYTES / 16); i += THREADS) c4[i] = make_uint4(0u, 0u, 0u, 0u);
  };
  uint32_t key[ITEMS], val[PAIRS ? ITEMS : 1];
  auto load_tile = [&](uint32_t t) {
    const size_t base = size_t(t) * TILE;
    const size_t wbase = base + size_t(warp) * 32 * ITEMS + lane;
    if (base + TILE <= size_t(a.n)) {
#pragma unroll
      for (int j = 0; j < ITEMS; ++j) key[j] = to_ordered(ld_stream(kin + wbase + j * 32), xin);
      if constexpr (PAIRS) {
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) val[j] = ld_stream(vin + wbase + j * 32);
      }
    } else {  // keys past the end act as 0xFFFFFFFF and sort to the tail
#pragma unroll
      for (int j = 0; j < ITEMS; ++j) {
        const size_t idx = wbase + j * 32;
        key[j] = idx < a.n ? to_ordered(kin[idx], xin) : 0xffffffffu;
        if constexpr (PAIRS) val[j] = idx < a.n ? vin[idx] : 0u;
      }
    }
  };
  // Write a staged tile out in tile order; runs of one digit go to
  // consecutive addresses.  The range check only guards against a corrupted
  // offset (error bit instead of an out-of-bounds write).
  auto write_out = [&](const uint32_t* buf, const uint32_t* goff, uint32_t valid) {
    bool oob = false;
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
      const uint32_t i = k * THREADS + tid;
      if (i < valid) {
        const uint32_t kk = buf[i];
        const uint32_t g = goff[digit_of(kk, shift, width)] + i;
        if (g < a.n) {
          kout[g] = from_ordered(kk, xout);
          if constexpr (PAIRS) vout[g] = buf[TILE + i];
        } else {
          oob = true;
        }
      }
    }
    if (oob) atomicOr(a.err, kErrBounds);
  };

  clear_tables();
  if (tid == 0) s_tile[0] = atomicAdd(a.tile_counter, 1u);
  __syncthreads();
  uint32_t t = s_tile[0];
  if (t >= num_tiles) return;
  load_tile(t);
  uint32_t prev_valid = 0;
  int it = 0;
  for (;;) {
    const size_t left = size_t(a.n) - size_t(t) * TILE;
    const uint32_t valid = left < size_t(TILE) ? uint32_t(left) : uint32_t(TILE);
    // rank within the warp
    uint32_t rk[(ITEMS + 1) / 2];
    warp_rank<R, ITEMS>(key, shift, width, s_mask + warp * kMaskSlots, s_cnt + warp * DIGITS, rk);
    __syncthreads();
    // per digit: tile count -> aggregate status; exclusive (digit, warp) prefixes
    uint32_t tot = 0, loff = 0;
    if (tid < DIGITS) {
#pragma unroll 4
      for (int wi = 0; wi < WARPS; ++wi) tot += s_cnt[wi * DIGITS + tid];
      st_relaxed(status + size_t(t) * DIGITS + tid, status_word<S>(parity, t == 0, tot));
    }
    const uint32_t excl = block_exclusive_sum<THREADS>(tid < DIGITS ? tot : 0u, s_warp);
    if (tid < DIGITS) {
      loff = excl;
      uint32_t run = excl;
#pragma unroll 4
      for (int wi = 0; wi < WARPS; ++wi) {
        const uint32_t v = s_cnt[wi * DIGITS + tid];
        s_cnt[wi * DIGITS + tid] = uint16_t(run);
        run += v;
      }
    }
    __syncthreads();
    // stage tile t in digit order
    uint32_t* buf = s_buf(it);
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      const uint32_t pos = ((rk[j >> 1] >> (16 * (j & 1))) & 0xffffu) + s_cnt[warp * DIGITS + digit_of(key[j], shift, width)];
      buf[pos] = key[j];
      if constexpr (PAIRS) buf[TILE + pos] = val[j];
    }
    __syncthreads();  // tables are dead, the staged tile is complete
    if (tid == 0) s_tile[1] = atomicAdd(a.tile_counter, 1u);
    clear_tables();
    __syncthreads();
    const uint32_t tn = s_tile[1];
    if (tn < num_tiles) load_tile(tn);  // prefetch the next tile's keys
    // first lookback window of t, then the previous tile's write-out
    DigitLookback<S, LB> lb;
    if (tid < DIGITS) {
      lb.start(t, 0);
      if (!lb.done) lb.issue(status, DIGITS, tid, 0);
    }
    if (it > 0) write_out(s_buf(it - 1), s_goff + ((it - 1) & 1) * DIGITS, prev_valid);
    if (tid < DIGITS) {
      while (!lb.done) {
        if (lb.consume(0, parity, a.err)) {
          if (lb.done) break;
        } else if (++lb.spins > kSpinLimit) {
          atomicOr(a.err, kErrTimeout);
          break;
        } else if (lb.spins > 16) {
          __nanosleep(100);
        }
        lb.issue(status, DIGITS, tid, 0);
      }
      if (t > 0) st_relaxed(status + size_t(t) * DIGITS + tid, status_word<S>(parity, true, lb.prefix + tot));
      s_goff[(it & 1) * DIGITS + tid] = a.bases[tid] + lb.prefix - loff;
    }
    __syncthreads();  // t's offsets are visible; the previous buffer is free
    prev_valid = valid;
    ++it;
    if (tn >= num_tiles) break;
    t = tn;
  }
  write_out(s_buf(it - 1), s_goff + ((it - 1) & 1) * DIGITS, prev_valid);
}

template <int R, int THREADS, int ITEMS, bool PAIRS, typename S, int MINB>
cudaError_t launch_onesweep_pipe(const PassArgs& a, unsigned grid, cudaStream_t s) {
  using L = PipeLayout<R, THREADS, ITEMS, PAIRS>;
  onesweep_pipe_kernel<R, THREADS, ITEMS, PAIRS, S, MINB><<<grid, THREADS, L::SMEM, s>>>(a);
  return cudaGetLastError();
}

template <int R, int THREADS, int ITEMS, bool PAIRS, typename S, int MINB>
OnesweepKernel make_onesweep_pipe(int shape_id) {
  using L = PipeLayout<R, THREADS, ITEMS, PAIRS>;
  OnesweepKernel k{R,
                   shape_id,
                   THREADS,
                   ITEMS,
                   L::TILE,
                   PAIRS,
                   sizeof(S) == 8,
                   L::SMEM,
                   &launch_onesweep_pipe<R, THREADS, ITEMS, PAIRS, S, MINB>,
                   reinterpret_cast<const void*>(&onesweep_pipe_kernel<R, THREADS, ITEMS, PAIRS, S, MINB>)};
  k.persistent_per_sm = MINB;
  return k;
}

}  // namespace rs
