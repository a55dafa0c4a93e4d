// The LSD distribution pass by an 8-bit digit with half-warp rank groups and
// early digit counts ("onesweep", second form).
//
// Paper: the same step as onesweep.cuh, the bucketing/distribution of
// Sec. 3.2 (count per bucket, cumulative totals, the partial sort grouping
// keys by bucket in ascending order, distribution of contiguous bucket
// ranges) done exactly, stable so that the repeated low-to-high passes sort
// (Sec. 3.3.1).  What differs is how a tile ranks its keys:
//
//  * Rank groups are half-warps.  Group g (warp w, half h) owns a contiguous
//    run of 16 * ITEMS keys of the tile: item j of its lane l is the run's
//    key j * 16 + l, so the group's keys in (item, lane) order are in input
//    order, and the groups' runs follow each other in input order.
//  * Early counts: every key first adds one to its group's counter for its
//    digit (a shared-memory reduction, no return value).  The tile's count
//    per digit is then known before any key is ranked: it is published as
//    the tile's aggregate status at once (so that successors' lookbacks
//    rarely wait), the digit threads scan it, and each (group, digit)
//    counter is replaced by the position, in the digit-sorted tile, of the
//    group's first key with that digit.
//  * One 32-bit word per (group, digit) holds [lane mask : 16 | position :
//    16].  Per item, each lane ORs its bit into the mask of its digit, reads
//    the word back (the lanes of its group with the same digit, and where
//    the run of that digit continues), and the highest such lane writes the
//    advanced position with the mask cleared: three shared-memory accesses
//    per key, after which the key's place in the staged tile is final and
//    it is staged right away.
//  * The digit threads (one per digit) run the lookback over earlier tiles
//    before ranking their own keys, so its latency overlaps the other
//    warps' ranking.
//
// Per tile (TILE = THREADS * ITEMS keys, tiles handed out by an atomic
// ticket so that every predecessor of a tile is already running):
//  1. load, 2. early counts, 3. per digit: aggregate status, scan, group
//  positions, 4. lookback (digit threads) and rank + stage (all), 5. stage
//  payloads (key+payload), 6. write out in tile order, each key to
//  base[digit] + (keys of the digit in earlier tiles) + (position within
//  the digit here).
#pragma once

#include "onesweep.cuh"

namespace rs {

template <int THREADS, int ITEMS, int NV>
struct Onesweep2Layout {
  static constexpr int DIGITS = 256;
  static constexpr int WARPS = THREADS / 32;
  static constexpr int GROUPS = 2 * WARPS;    // half-warp rank groups
  static constexpr int TILE = THREADS * ITEMS;
  static constexpr int GKEYS = 16 * ITEMS;    // keys of one group
  static constexpr size_t KBUF = size_t(TILE) * 4;                 // staged keys
  // A group's row of rank words is one word longer than the digits, so that
  // the same digit in the two halves of a warp (rows g and g + 1) falls in
  // adjacent banks instead of one: keys with few distinct digits (clustered
  // values, runs of equal keys) otherwise make the halves' accesses to a
  // digit collide in its bank (2^26 keys in 8 clusters: 96 M shared-memory
  // wavefronts per pass instead of 48 M).
  static constexpr int ROW = DIGITS + 1;
  static constexpr size_t TBL = size_t(GROUPS) * ROW * 4;          // [GROUPS][ROW] rank words
  // The rank words sit after the staged keys; with a payload they share
  // their space with the staged payloads, which are written only after the
  // last rank word is read.
  static constexpr size_t OFF_TBL = KBUF;
  static constexpr size_t END = (KBUF + TBL > KBUF * (1 + NV) ? KBUF + TBL : KBUF * (1 + NV));
  static constexpr size_t OFF_GOFF = (END + 15) / 16 * 16;
  static constexpr size_t OFF_SCAN = OFF_GOFF + size_t(DIGITS) * 4;
  static constexpr size_t OFF_TILE = OFF_SCAN + 32 * 4;
  static constexpr size_t SMEM = OFF_TILE + 16;
  static_assert(THREADS % 32 == 0 && THREADS >= DIGITS && THREADS <= 1024, "one thread per digit at least");
  static_assert(TILE < 65536, "positions are 16-bit");
  static_assert(TBL % 16 == 0, "the rank words are cleared as 16-byte vectors");
  static_assert(SMEM <= 227 * 1024, "shared memory");
};

// 32-bit shared-memory accesses by address (the hot loop's tables).
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void sh_red_add(uint32_t a, uint32_t v) {
  asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void sh_red_or(uint32_t a, uint32_t v) {
  asm volatile("red.shared.or.b32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t sh_ld(uint32_t a) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ void sh_st(uint32_t a, uint32_t v) {
  asm volatile("st.shared.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void st_global(uint32_t* p, uint32_t v) {
  asm volatile("st.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Byte `sel & 3` of k as the low byte of the result (a byte permute with the
// upper three bytes taken from zero): the 8-bit digit at shift 8 * (sel & 3).
__device__ __forceinline__ uint32_t byte_digit(uint32_t k, uint32_t sel) { return __byte_perm(k, 0u, sel); }

// Exclusive prefix sum over the first 256 threads of the block (8 warps),
// synchronised by named barrier 1; s_scan holds 8 words.
__device__ __forceinline__ uint32_t scan256_exclusive(uint32_t x, uint32_t* s_scan) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) s_scan[w] = inc;
  asm volatile("bar.sync 1, 256;" ::: "memory");
  uint32_t before = 0;
#pragma unroll
  for (int i = 0; i < 7; ++i)
    if (i < w) before += s_scan[i];
  return before + inc - x;
}

// Where one tile of a pass comes from and goes to (the pass kernel fills it
// from its launch arguments and its ticket; the single-launch sort from its
// own plan of passes).
struct Tile2Job {
  uint32_t tile;         // tile index (row of the status array)
  uint32_t n;            // keys of the pass
  const uint32_t* kin;
  uint32_t* kout;
  const uint32_t* vin;   // payloads (NV >= 1)
  uint32_t* vout;
  KeyXform xin, xout;    // applied on load / inverted on store
  uint32_t parity;       // status parity of this pass
  void* status;          // [tiles][256] status words
  const uint32_t* bases; // [256] keys with a smaller digit (global or shared memory)
  uint32_t shift;        // the digit is byte shift / 8 of the key
  uint32_t* err;         // device error word
};

// A key or payload load: read-only path for pass kernels; coherent (L2) in
// the single-launch sort, whose later passes read what other blocks of the
// same launch wrote.
template <bool COHERENT>
__device__ __forceinline__ uint32_t ld_pass(const uint32_t* p) {
  if constexpr (COHERENT) {
    uint32_t v;
    asm volatile("ld.global.cg.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
  } else {
    return ld_stream(p);
  }
}

// Steps 1-6 for one tile.  The rank words must be zero and the block
// synchronised on entry; the block is synchronised on return.
// UNSTABLE (keys only): the first executed pass, see step 2u.
template <int THREADS, int ITEMS, int NV, typename S, bool EARLY_LB, int LB, bool COHERENT, bool UNSTABLE = false>
__device__ __forceinline__ void onesweep2_tile(const Tile2Job& job, unsigned char* smem) {
  using L = Onesweep2Layout<THREADS, ITEMS, NV>;
  constexpr int DIGITS = L::DIGITS, GROUPS = L::GROUPS, TILE = L::TILE;
  uint32_t* s_key = reinterpret_cast<uint32_t*>(smem);
  uint32_t* s_val = reinterpret_cast<uint32_t*>(smem + L::KBUF);
  uint32_t* s_tbl = reinterpret_cast<uint32_t*>(smem + L::OFF_TBL);
  uint32_t* s_goff = reinterpret_cast<uint32_t*>(smem + L::OFF_GOFF);
  uint32_t* s_scan = reinterpret_cast<uint32_t*>(smem + L::OFF_SCAN);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int l16 = lane & 15, grp = warp * 2 + (lane >> 4);
  const uint32_t tile = job.tile;
  const uint32_t* kin = job.kin;
  uint32_t* kout = job.kout;
  const uint32_t* vin = job.vin;
  uint32_t* vout = job.vout;
  const KeyXform xin = job.xin, xout = job.xout;
  const uint32_t parity = job.parity;
  S* status = reinterpret_cast<S*>(job.status);
  const size_t tbase = size_t(tile) * TILE;
  const size_t left = size_t(job.n) - tbase;
  // UNSTABLE runs on full tiles only: keys past the end would take places
  // among the tile's real keys of digit 255 (the atomic ranking keeps no
  // order), so the caller gives a partial tile to the stable body
  const uint32_t valid = (NV == 0 && UNSTABLE) || left >= size_t(TILE) ? uint32_t(TILE) : uint32_t(left);
  const uint32_t sel = 0x4440u | (job.shift >> 3);
  (void)vin;
  (void)vout;
  (void)s_val;

  // 1p. the payload words of a full tile, prefetched into L2 for step 5
  if constexpr (NV >= 1) {
    if (valid == TILE && (reinterpret_cast<uintptr_t>(vin + tbase) & 15u) == 0)
      prefetch_l2_tile(vin + tbase, uint32_t(TILE) * 4u);
  }

  // 1. load: group grp takes keys [grp * GKEYS, (grp + 1) * GKEYS) of the
  // tile, item j of lane l16 being key grp * GKEYS + j * 16 + l16.  Keys
  // past the end act as 0xFFFFFFFF: their digit is the largest and they
  // come after every real key, so they sort to the tile's tail and are
  // never written.
  uint32_t key[ITEMS];
  const uint32_t goff_in = uint32_t(grp) * L::GKEYS + uint32_t(l16);
  if (valid == TILE) {
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) key[j] = ld_pass<COHERENT>(kin + tbase + goff_in + j * 16);
    if (!is_identity(xin)) {
#pragma unroll
      for (int j = 0; j < ITEMS; ++j) key[j] = to_ordered(key[j], xin);
    }
  } else {
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      const uint32_t i = goff_in + j * 16;
      key[j] = i < valid ? to_ordered(ld_pass<COHERENT>(kin + tbase + i), xin) : 0xffffffffu;
    }
  }

  // Keys only, first executed pass of a full tile (UNSTABLE): the order of
  // keys with the same lowest digit is free (there is no earlier order to
  // keep, and keys with equal digits here are told apart by the later passes
  // or are equal), so one shared counter per (half of a warp, digit)
  // suffices and a key's position is one atomic add on it (steps 2u and 4u
  // below) instead of the groups' mask words.  Two rows, one per half, keep
  // the halves' accesses to one digit in different banks.
  constexpr bool unstable = NV == 0 && UNSTABLE;

  // 2. early counts per (group, digit) [2u: per (half, digit)]
  const uint32_t tb_grp = smem_addr(s_tbl + (unstable ? (lane >> 4) : grp) * L::ROW);
#pragma unroll
  for (int j = 0; j < ITEMS; ++j) sh_red_add(tb_grp + 4u * byte_digit(key[j], sel), 1u);
  __syncthreads();

  // 3. per digit (threads 0..255): the tile's count -> aggregate status now;
  // exclusive scan over digits -> where each digit's run starts in the
  // staged tile; then each group's counter -> the position of its first key
  // of the digit [3u: the two halves' counters -> where each half's keys of
  // the digit start]
  uint32_t tot = 0, excl = 0;
  if (tid < DIGITS) {
    if constexpr (unstable) {
      tot = s_tbl[tid] + s_tbl[L::ROW + tid];
    } else {
#pragma unroll 8
      for (int g = 0; g < GROUPS; ++g) tot += s_tbl[g * L::ROW + tid];
    }
    st_relaxed(status + size_t(tile) * DIGITS + tid, status_word<S>(parity, tile == 0, tot));
    excl = scan256_exclusive(tot, s_scan);
    if constexpr (unstable) {
      const uint32_t c0 = s_tbl[tid];
      s_tbl[tid] = excl;
      s_tbl[L::ROW + tid] = excl + c0;
    } else {
      uint32_t run = excl;
#pragma unroll 8
      for (int g = 0; g < GROUPS; ++g) {
        const uint32_t c = s_tbl[g * L::ROW + tid];
        s_tbl[g * L::ROW + tid] = run;
        run += c;
      }
    }
  }
  __syncthreads();

  // 4a. lookback over earlier tiles (digit threads): publishes this tile's
  // inclusive counts and the digit's output offset for the write-out.  Run
  // before the digit threads rank their own keys (EARLY_LB), it overlaps the
  // other warps' ranking; after, it needs fewer live registers.
  auto do_lookback = [&]() {
    if (tid < DIGITS) {
      uint32_t prefix[1];
      lookback<DIGITS, 1, S, LB>(status, tile, 0u, tid, parity, job.err, prefix);
      if (tile != 0) st_relaxed(status + size_t(tile) * DIGITS + tid, status_word<S>(parity, true, prefix[0] + tot));
      s_goff[tid] = job.bases[tid] + prefix[0] - excl;
    }
  };
  if constexpr (EARLY_LB) do_lookback();

  // 4b. rank within the group and stage the key at its final tile position
  const uint32_t lt16 = (1u << l16) - 1u;
  const uint32_t mybit = 1u << (16 + l16);
  const uint32_t sk = smem_addr(s_key);
  uint32_t pos[NV >= 1 ? (ITEMS + 1) / 2 : 1];
  if constexpr (unstable) {
    // 4u. one atomic add per key on its digit's counter gives its place
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      uint32_t p;
      asm volatile("atom.shared.add.u32 %0, [%1], 1;" : "=r"(p) : "r"(tb_grp + 4u * byte_digit(key[j], sel)) : "memory");
      sh_st(sk + 4u * p, key[j]);
    }
  } else {
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      const uint32_t ad = tb_grp + 4u * byte_digit(key[j], sel);
      sh_red_or(ad, mybit);
      __syncwarp();
      const uint32_t v = sh_ld(ad);
      const uint32_t peers = v >> 16, base = v & 0xffffu;
      const uint32_t p = base + __popc(peers & lt16);
      if ((peers >> l16) == 1u) sh_st(ad, base + __popc(peers));  // the group's highest lane with this digit
      __syncwarp();
      sh_st(sk + 4u * p, key[j]);
      if constexpr (NV >= 1) {
        if (j & 1) pos[j >> 1] |= p << 16;
        else pos[j >> 1] = p;
      }
    }
  }
  if constexpr (!EARLY_LB) do_lookback();
  __syncthreads();

  // 5. payloads: staged at their keys' positions (over the dead rank words)
  if constexpr (NV >= 1) {
    uint32_t val[ITEMS];
    if (valid == TILE) {
#pragma unroll
      for (int j = 0; j < ITEMS; ++j) val[j] = ld_pass<COHERENT>(vin + tbase + goff_in + j * 16);
    } else {
#pragma unroll
      for (int j = 0; j < ITEMS; ++j) {
        const uint32_t i = goff_in + j * 16;
        val[j] = i < valid ? ld_pass<COHERENT>(vin + tbase + i) : 0u;
      }
    }
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) s_val[(pos[j >> 1] >> (16 * (j & 1))) & 0xffffu] = val[j];
    __syncthreads();
  }

  // 6. write out in tile order: runs of one digit go to consecutive
  // addresses.  Keys are read from shared memory and their offsets looked up
  // a batch at a time before the batch's stores, so that the stores (global,
  // through an explicit global-space instruction) do not serialise the
  // shared-memory loads behind them (GB300, 2^26 keys: the write-out of a
  // 512 x 24 tile went from about 8,300 to 5,100 SM cycles).  The range
  // check only guards against a corrupted offset (it raises an error bit
  // instead of writing out of bounds).
  bool oob = false;
  const uint32_t n = job.n;
  const uint32_t sg = smem_addr(s_goff);
  auto write_out = [&](auto invert) {
    constexpr int B = ITEMS % 8 == 0 ? 8 : (ITEMS % 6 == 0 ? 6 : (ITEMS % 4 == 0 ? 4 : 1));
#pragma unroll
    for (int k0 = 0; k0 < ITEMS; k0 += B) {
      uint32_t kk[B], g[B];
#pragma unroll
      for (int b = 0; b < B; ++b) kk[b] = sh_ld(sk + 4u * ((k0 + b) * THREADS + tid));
#pragma unroll
      for (int b = 0; b < B; ++b) g[b] = sh_ld(sg + 4u * byte_digit(kk[b], sel)) + (k0 + b) * THREADS + tid;
#pragma unroll
      for (int b = 0; b < B; ++b) {
        const uint32_t i = (k0 + b) * THREADS + tid;
        if (valid == TILE || i < valid) {
          if (g[b] < n) {
            st_global(kout + g[b], decltype(invert)::value ? from_ordered(kk[b], xout) : kk[b]);
            if constexpr (NV >= 1) st_global(vout + g[b], sh_ld(smem_addr(s_val) + 4u * i));
          } else {
            oob = true;
          }
        }
      }
    }
  };
  if (is_identity(xout)) write_out(std::false_type{});
  else write_out(std::true_type{});
  if (oob) atomicOr(job.err, kErrBounds);
  __syncthreads();
}


template <int THREADS, int ITEMS, int NV, typename S, int MINB, bool EARLY_LB, int LB, bool UNSTABLE>
__global__ void __launch_bounds__(THREADS, MINB) onesweep2_kernel(const PassArgs a) {
  using L = Onesweep2Layout<THREADS, ITEMS, NV>;
  extern __shared__ __align__(16) unsigned char smem[];
  const Route route = route_of(a.skip, a.pass, a.num_passes);
  if (!route.active) return;
  Tile2Job job;
  job.kin = route.src == BUF_IN ? a.keys_in : (route.src == BUF_OUT ? a.keys_out : a.keys_alt);
  job.kout = route.dst == BUF_OUT ? a.keys_out : a.keys_alt;
  job.vin = nullptr;
  job.vout = nullptr;
  if constexpr (NV >= 1) {
    job.vin = route.src == BUF_IN ? a.vals_in : (route.src == BUF_OUT ? a.vals_out : a.vals_alt);
    job.vout = route.dst == BUF_OUT ? a.vals_out : a.vals_alt;
  }
  job.xin = route.src == BUF_IN ? a.xin : KeyXform{0u, 0u};
  job.xout = route.last ? a.xout : KeyXform{0u, 0u};
  job.parity = route.parity;
  job.status = a.status;
  job.bases = a.bases;
  job.shift = a.shift;
  job.err = a.err;
  job.n = a.n;
  // 0. clear the rank words, take the tile ticket
  uint32_t* s_tile = reinterpret_cast<uint32_t*>(smem + L::OFF_TILE);
  {
    uint4* t4 = reinterpret_cast<uint4*>(smem + L::OFF_TBL);
#pragma unroll 4
    for (int i = threadIdx.x; i < int(L::TBL / 16); i += THREADS) t4[i] = make_uint4(0u, 0u, 0u, 0u);
    if (threadIdx.x == 0) *s_tile = atomicAdd(a.tile_counter, 1u);
  }
  __syncthreads();
  job.tile = *s_tile;
  if constexpr (UNSTABLE) {
    // the first executed pass of this sort, on a full tile
    if (route.src == BUF_IN && (size_t(job.tile) + 1) * L::TILE <= size_t(a.n)) {
      onesweep2_tile<THREADS, ITEMS, NV, S, EARLY_LB, LB, false, true>(job, smem);
      return;
    }
  }
  onesweep2_tile<THREADS, ITEMS, NV, S, EARLY_LB, LB, false, false>(job, smem);
}

template <int THREADS, int ITEMS, int NV, typename S, int MINB, bool EARLY_LB, int LB, bool UNSTABLE>
cudaError_t launch_onesweep2(const PassArgs& a, unsigned grid, cudaStream_t s) {
  using L = Onesweep2Layout<THREADS, ITEMS, NV>;
  onesweep2_kernel<THREADS, ITEMS, NV, S, MINB, EARLY_LB, LB, UNSTABLE><<<grid, THREADS, L::SMEM, s>>>(a);
  return cudaGetLastError();
}

// EARLY_LB: the digit threads run the lookback before ranking their keys;
// LB: predecessors' status words a digit thread reads per lookback round.
template <int THREADS, int ITEMS, int NV, typename S, int MINB, bool EARLY_LB = false, int LB = 8>
OnesweepKernel make_onesweep2(int shape_id) {
  using L = Onesweep2Layout<THREADS, ITEMS, NV>;
  cudaError_t (*first)(const PassArgs&, unsigned, cudaStream_t) = nullptr;
  const void* first_func = nullptr;
  if constexpr (NV == 0) {
    first = &launch_onesweep2<THREADS, ITEMS, NV, S, MINB, EARLY_LB, LB, true>;
    first_func = reinterpret_cast<const void*>(&onesweep2_kernel<THREADS, ITEMS, NV, S, MINB, EARLY_LB, LB, true>);
  }
  return OnesweepKernel{8,
                        shape_id,
                        THREADS,
                        ITEMS,
                        L::TILE,
                        NV >= 1,
                        sizeof(S) == 8,
                        L::SMEM,
                        &launch_onesweep2<THREADS, ITEMS, NV, S, MINB, EARLY_LB, LB, false>,
                        reinterpret_cast<const void*>(&onesweep2_kernel<THREADS, ITEMS, NV, S, MINB, EARLY_LB, LB, false>),
                        0,
                        NV,
                        false,
                        first,
                        first_func};
}

}  // namespace rs
