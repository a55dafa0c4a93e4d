// Device helpers shared by the sort kernels (sm_103a).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "rs_internal.h"

namespace rs {

// Rounds of the cross-tile lookback a tile waits on a predecessor that has
// not published yet before it gives up and raises the device error word.
// A round is at least one L2 round trip plus a 100 ns sleep, so the limit is
// tens of milliseconds, far above the microseconds a predecessor needs.
constexpr uint32_t kSpinLimit = 1u << 16;
// Bits of the device error word.
constexpr uint32_t kErrTimeout = 1u;  // a bounded wait gave up
constexpr uint32_t kErrBounds = 2u;   // a computed output index was out of range (skipped)

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ uint32_t lanemask_gt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_gt;" : "=r"(m));
  return m;
}

// The order-preserving map of KeyXform and its inverse (the inverse looks at
// the mapped word's top bit, which is the complement of the key's sign).
__device__ __forceinline__ uint32_t to_ordered(uint32_t k, KeyXform x) {
  return k ^ ((uint32_t(int32_t(k) >> 31) & x.fmask) ^ x.smask);
}
__device__ __forceinline__ uint32_t from_ordered(uint32_t t, KeyXform x) {
  return t ^ ((uint32_t(~int32_t(t) >> 31) & x.fmask) ^ x.smask);
}
__host__ __device__ __forceinline__ bool is_identity(KeyXform x) { return (x.fmask | x.smask) == 0u; }

// The same map for 64-bit keys held as (low, high) words: the sign is the top
// bit of the high word, and a set sign flips the low word by flo.
__device__ __forceinline__ uint2 map64(uint2 k, KeyXform64 x) {
  const uint32_t neg = uint32_t(int32_t(k.y) >> 31);  // all ones for a set sign bit
  return make_uint2(k.x ^ (neg & x.flo), k.y ^ ((neg & x.fhi) ^ x.shi));
}
__device__ __forceinline__ uint2 unmap64(uint2 t, KeyXform64 x) {
  const uint32_t neg = uint32_t(~int32_t(t.y) >> 31);  // the original sign is the complement of the top bit
  return make_uint2(t.x ^ (neg & x.flo), t.y ^ ((neg & x.fhi) ^ x.shi));
}

// Digit of `width` bits at `shift` (1 <= width <= 31, shift + width <= 32):
// a shift and a mask (the mask is loop-invariant and hoisted by the compiler;
// a bit-field extract with run-time operands takes more instructions).
__device__ __forceinline__ uint32_t digit_of(uint32_t key, uint32_t shift, uint32_t width) {
  return (key >> shift) & ((1u << width) - 1u);
}

// ---- relaxed, gpu-scope accesses for the cross-tile status words ----------
__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed(uint32_t* p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// ---- L2 prefetch of a tile's payloads ---------------------------------------
// The pass kernels load a tile's payload words only after ranking its keys;
// asking the TMA unit at the start of the tile to bring them into L2 turns
// that load's DRAM latency into an L2 hit.  Threads 0.. of the block each
// issue one bulk prefetch of up to kPrefetchPiece bytes (a hint: nothing to
// wait for).  p must be 16-byte aligned and bytes a multiple of 16.
constexpr uint32_t kPrefetchPiece = 4096;
__device__ __forceinline__ void prefetch_l2_tile(const void* p, uint32_t bytes) {
  const uint32_t off = threadIdx.x * kPrefetchPiece;
  if (off < bytes) {
    const uint32_t len = bytes - off < kPrefetchPiece ? bytes - off : kPrefetchPiece;
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(static_cast<const char*>(p) + off), "r"(len)
                 : "memory");
  }
}

// ---- streaming global accesses for keys and payloads ----------------------
// Keys are read once per pass: keep them out of L1.
__device__ __forceinline__ uint32_t ld_stream(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.global.nc.L1::no_allocate.u32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ uint2 ld_stream2(const uint2* p) {
  uint2 v;
  asm volatile("ld.global.nc.L1::no_allocate.v2.u32 {%0,%1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p));
  return v;
}
__device__ __forceinline__ uint4 ld_stream4(const uint4* p) {
  uint4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}

// ---- the status word of one (tile, digit) of the chained scan --------------
// Layout, most significant first: [parity][inclusive][count].  `parity`
// tells the passes of one sort apart without re-zeroing the array between
// passes: executed pass i writes parity (i & 1) ^ 1, so words left over from
// the pass before (or zeroes, for the first) never look ready.  `inclusive`
// marks a count that already includes every earlier tile.
template <typename S>
struct StatusCodec;
template <>
struct StatusCodec<uint32_t> {
  static constexpr uint32_t kPar = 1u << 31;
  static constexpr uint32_t kInc = 1u << 30;
  static constexpr uint32_t kVal = kInc - 1;
};
template <>
struct StatusCodec<unsigned long long> {
  static constexpr unsigned long long kPar = 1ull << 63;
  static constexpr unsigned long long kInc = 1ull << 62;
  static constexpr unsigned long long kVal = kInc - 1;
};

template <typename S>
__device__ __forceinline__ S status_word(uint32_t parity, bool inclusive, uint32_t count) {
  using C = StatusCodec<S>;
  return (parity ? C::kPar : S(0)) | (inclusive ? C::kInc : S(0)) | S(count);
}
template <typename S>
__device__ __forceinline__ bool status_ready(S w, uint32_t parity) {
  return ((w & StatusCodec<S>::kPar) != 0) == (parity != 0);
}
template <typename S>
__device__ __forceinline__ bool status_inclusive(S w) {
  return (w & StatusCodec<S>::kInc) != 0;
}
template <typename S>
__device__ __forceinline__ uint32_t status_count(S w) {
  return uint32_t(w & StatusCodec<S>::kVal);
}

// ---- block-wide exclusive prefix sum ---------------------------------------
// Every thread of the block must call it.  s_warp holds THREADS/32 words.
template <int THREADS>
__device__ __forceinline__ uint32_t block_exclusive_sum(uint32_t x, uint32_t* s_warp,
                                                        uint32_t* total = nullptr) {
  constexpr int WARPS = THREADS / 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) s_warp[w] = inc;
  __syncthreads();
  if (w == 0) {
    uint32_t t = lane < WARPS ? s_warp[lane] : 0u;
    uint32_t ti = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, ti, o);
      if (lane >= o) ti += y;
    }
    if (lane < WARPS) s_warp[lane] = ti - t;  // exclusive warp offsets
    if (lane == WARPS - 1 && total) *total = ti;
  }
  __syncthreads();
  uint32_t r = s_warp[w] + inc - x;
  __syncthreads();  // s_warp may be reused by the caller
  return r;
}

// ---- which buffers an LSD pass reads and writes -----------------------------
enum : int { BUF_IN = 0, BUF_OUT = 1, BUF_ALT = 2 };
struct Route {
  int active;
  int src, dst;
  int last;  // the last executed pass (it writes the final order into keys_out)
  uint32_t parity;
};

// Passes whose digit is skippable (one bucket holds every key) do not run.
// The executed passes alternate between keys_out and the alternate buffer so
// that the last one lands in keys_out; the first reads the input.  If every
// digit is skippable the last pass still runs (it is then a stable identity
// copy into keys_out).  `skip` may be null (no pass skipped).
__device__ __forceinline__ Route route_of(const uint32_t* skip, int pass, int num_passes) {
  int m = 0, idx = -1;
  for (int p = 0; p < num_passes; ++p) {
    const bool s = skip ? skip[p] != 0 : false;
    if (!s) {
      if (p == pass) idx = m;
      ++m;
    }
  }
  if (m == 0) {
    m = 1;
    if (pass == num_passes - 1) idx = 0;
  }
  Route r;
  r.active = idx >= 0;
  if (!r.active) {
    r.src = r.dst = BUF_IN;
    r.last = 0;
    r.parity = 0;
    return r;
  }
  r.last = idx == m - 1;
  r.dst = ((m - 1 - idx) % 2 == 0) ? BUF_OUT : BUF_ALT;
  r.src = idx == 0 ? BUF_IN : (((m - idx) % 2 == 0) ? BUF_OUT : BUF_ALT);
  r.parity = uint32_t(idx & 1) ^ 1u;
  return r;
}

}  // namespace rs
