// Upfront digit histograms (every digit in one read of the keys) and their
// exclusive scans.
//
// Paper: the count loop of the bucketing phase, where each element adds one
// to the counter of its bucket (Sec. 3.2), here over every digit of the keys'
// order-preserving unsigned map, followed by the cumulative totals (Sec. 3.2;
// Sec. 4.4 sums the per-cell totals after making them cumulative).  On the
// AP1000 each cell counted its own elements and a hypercube summation added
// the 64 arrays (Sec. 4.4); here each block counts a slice of the keys into
// shared memory and the block arrays are added into one global array.
#include "rs_device.cuh"
#include "rs_internal.h"

namespace rs {

// Block-private sub-histograms per digit; warps are spread over COPIES
// copies to thin out shared-memory atomic collisions on skewed data.
template <int R, int THREADS, int COPIES, bool XF>
__global__ void __launch_bounds__(THREADS) upfront_hist_kernel(const HistArgs a) {
  constexpr int DIGITS = 1 << R;
  extern __shared__ __align__(16) uint32_t sh[];  // [COPIES][num_digits][DIGITS]
  const int nd = a.num_digits;
  const int tid = threadIdx.x;
  const int per_copy = nd * DIGITS;
  for (int i = tid; i < COPIES * per_copy; i += THREADS) sh[i] = 0u;
  __syncthreads();
  uint32_t* my = sh + ((tid >> 5) % COPIES) * per_copy;

  uint32_t sft[kMaxDigits], wid[kMaxDigits];
#pragma unroll
  for (int j = 0; j < kMaxDigits; ++j) {
    sft[j] = a.dig[j].shift;
    wid[j] = a.dig[j].width;
  }
  const KeyXform xf = a.xform;
  auto count = [&](uint32_t k) {
    if constexpr (XF) k = to_ordered(k, xf);
#pragma unroll
    for (int j = 0; j < kMaxDigits; ++j)
      if (j < nd) atomicAdd(&my[j * DIGITS + digit_of(k, sft[j], wid[j])], 1u);
  };

  // keys before the first 16-byte boundary and after the last full vector
  const uint32_t n = a.n;
  const uint32_t mis = uint32_t((reinterpret_cast<uintptr_t>(a.keys) >> 2) & 3u);
  uint32_t head = (4u - mis) & 3u;
  if (head > n) head = n;
  const size_t nvec = size_t(n - head) / 4;
  const uint32_t tail = head + uint32_t(nvec * 4);
  if (blockIdx.x == gridDim.x - 1) {
    for (uint32_t i = tid; i < head; i += THREADS) count(a.keys[i]);
    for (uint32_t i = tail + tid; i < n; i += THREADS) count(a.keys[i]);
  }
  const uint4* v4 = reinterpret_cast<const uint4*>(a.keys + head);
  const size_t stride = size_t(gridDim.x) * THREADS;
  size_t i = size_t(blockIdx.x) * THREADS + tid;
  for (; i + 3 * stride < nvec; i += 4 * stride) {
    const uint4 x0 = ld_stream4(v4 + i);
    const uint4 x1 = ld_stream4(v4 + i + stride);
    const uint4 x2 = ld_stream4(v4 + i + 2 * stride);
    const uint4 x3 = ld_stream4(v4 + i + 3 * stride);
    count(x0.x); count(x0.y); count(x0.z); count(x0.w);
    count(x1.x); count(x1.y); count(x1.z); count(x1.w);
    count(x2.x); count(x2.y); count(x2.z); count(x2.w);
    count(x3.x); count(x3.y); count(x3.z); count(x3.w);
  }
  for (; i < nvec; i += stride) {
    const uint4 x = ld_stream4(v4 + i);
    count(x.x); count(x.y); count(x.z); count(x.w);
  }

  // clear the chained-scan status words for the passes that follow
  for (size_t z = size_t(blockIdx.x) * THREADS + tid; z < a.zero_vec4; z += stride)
    a.zero_ptr[z] = make_uint4(0u, 0u, 0u, 0u);

  __syncthreads();
  for (int b = tid; b < per_copy; b += THREADS) {
    uint32_t s = 0;
#pragma unroll
    for (int c = 0; c < COPIES; ++c) s += sh[c * per_copy + b];
    if (s) atomicAdd(&a.hist[b], s);
  }
}

// 8-bit digits: every lane of the block counts into its own copy of the
// histograms, laid out [digit][bin][lane] so that lane l only ever touches
// shared-memory bank l.  No atomic ever conflicts with another (not even when
// every key has the same digit), so the kernel runs at the speed of its
// loads.  Copies of one warp-lane position are shared by the block's warps
// (atomics still needed), 128 KiB of shared memory for four digits.
// BYTES: the four digits are the key's bytes (shift 8j, width 8), the plan of
// every 32-bit LSD sort with 8-bit digits.  The kernel is bound by its integer
// instructions, so this case takes each digit with one byte permute and
// counts it with one shift-add and one shared-memory reduction on a 32-bit
// shared address (about 13 instructions per key instead of 38).
template <int THREADS, bool XF, bool BYTES>
__global__ void __launch_bounds__(THREADS, 1) upfront_hist_lanes_kernel(const HistArgs a) {
  constexpr int BINS = 256;
  extern __shared__ __align__(16) uint32_t sh[];  // [num_digits][256][32]
  const int nd = a.num_digits;
  const int tid = threadIdx.x, lane = tid & 31;
  for (int i = tid; i < nd * BINS * 32; i += THREADS) sh[i] = 0u;
  __syncthreads();
  uint32_t sft[kMaxDigits], wid[kMaxDigits];
#pragma unroll
  for (int j = 0; j < kMaxDigits; ++j) {
    sft[j] = a.dig[j].shift;
    wid[j] = a.dig[j].width;
  }
  const KeyXform xf = a.xform;
  // this lane's copy of bin 0 of digit 0; a (digit j, bin b) counter is
  // BINS * 32 * 4 * j + 128 * b bytes further
  const uint32_t lane_base = uint32_t(__cvta_generic_to_shared(sh)) + uint32_t(lane) * 4u;
  auto count = [&](uint32_t k) {
    if constexpr (XF) k = to_ordered(k, xf);
    if constexpr (BYTES) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint32_t b = __byte_perm(k, 0u, 0x4440u + uint32_t(j));
        const uint32_t addr = lane_base + uint32_t(j * BINS * 32 * 4) + b * 128u;
        asm volatile("red.shared.add.u32 [%0], 1;" ::"r"(addr) : "memory");
      }
    } else {
#pragma unroll
      for (int j = 0; j < kMaxDigits; ++j)
        if (j < nd) atomicAdd(&sh[(j * BINS + digit_of(k, sft[j], wid[j])) * 32 + lane], 1u);
    }
  };
  const uint32_t n = a.n;
  const size_t stride = size_t(gridDim.x) * THREADS;
  const uint32_t mis = uint32_t((reinterpret_cast<uintptr_t>(a.keys) >> 2) & 3u);
  uint32_t head = (4u - mis) & 3u;
  if (head > n) head = n;
  const size_t nvec = size_t(n - head) / 4;
  const uint32_t tail = head + uint32_t(nvec * 4);
  if (blockIdx.x == gridDim.x - 1) {
    for (uint32_t i = tid; i < head; i += THREADS) count(a.keys[i]);
    for (uint32_t i = tail + tid; i < n; i += THREADS) count(a.keys[i]);
  }
  const uint4* v4 = reinterpret_cast<const uint4*>(a.keys + head);
  size_t i = size_t(blockIdx.x) * THREADS + tid;
  for (; i + 3 * stride < nvec; i += 4 * stride) {
    const uint4 x0 = ld_stream4(v4 + i);
    const uint4 x1 = ld_stream4(v4 + i + stride);
    const uint4 x2 = ld_stream4(v4 + i + 2 * stride);
    const uint4 x3 = ld_stream4(v4 + i + 3 * stride);
    count(x0.x); count(x0.y); count(x0.z); count(x0.w);
    count(x1.x); count(x1.y); count(x1.z); count(x1.w);
    count(x2.x); count(x2.y); count(x2.z); count(x2.w);
    count(x3.x); count(x3.y); count(x3.z); count(x3.w);
  }
  for (; i < nvec; i += stride) {
    const uint4 x = ld_stream4(v4 + i);
    count(x.x); count(x.y); count(x.z); count(x.w);
  }
  for (size_t z = size_t(blockIdx.x) * THREADS + tid; z < a.zero_vec4; z += stride)
    a.zero_ptr[z] = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();
  // one row of 32 lane copies per (digit, bin); each thread starts its row at
  // its own lane so that a warp's reads spread over all banks
  for (int b = tid; b < nd * BINS; b += THREADS) {
    uint32_t s = 0;
#pragma unroll 8
    for (int k = 0; k < 32; ++k) s += sh[b * 32 + ((k + lane) & 31)];
    if (s) atomicAdd(&a.hist[b], s);
  }
}

// All eight byte digits of interleaved 64-bit keys (their order map x64) in
// one read: digits 0-3 from the low word, 4-7 from the high word.  Eight
// digits with a copy per lane would take 256 KiB, so lanes l and l + 16 share
// a copy ([digit][bin][16]: 128 KiB); a shared copy costs a two-way bank
// conflict when the two lanes' bins differ and have the same parity.
constexpr int kHist64Threads = 1024;
constexpr size_t kHist64Smem = size_t(8) * 256 * 16 * 4;

__global__ void __launch_bounds__(kHist64Threads, 1) upfront_hist64_kernel(const HistArgs a) {
  extern __shared__ __align__(16) uint32_t sh[];  // [8][256][16]
  const int tid = threadIdx.x, lane = tid & 31;
  for (int i = tid; i < 8 * 256 * 16; i += kHist64Threads) sh[i] = 0u;
  __syncthreads();
  // this lane's copy of bin 0 of digit 0; (digit j, bin b) is 16 KiB * j + 64 * b bytes further
  const uint32_t base = uint32_t(__cvta_generic_to_shared(sh)) + uint32_t(lane & 15) * 4u;
  const KeyXform64 x64 = a.x64;
  auto count = [&](uint32_t lo, uint32_t hi) {
    const uint2 m = map64(make_uint2(lo, hi), x64);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const uint32_t b = __byte_perm(j < 4 ? m.x : m.y, 0u, 0x4440u + uint32_t(j & 3));
      const uint32_t addr = base + uint32_t(j * 256 * 16 * 4) + b * 64u;
      asm volatile("red.shared.add.u32 [%0], 1;" ::"r"(addr) : "memory");
    }
  };
  const uint32_t n = a.n;
  const size_t stride = size_t(gridDim.x) * kHist64Threads;
  // one key before the first 16-byte boundary, one after the last pair
  const uint32_t head = ((reinterpret_cast<uintptr_t>(a.keys64) >> 3) & 1u) && n > 0 ? 1u : 0u;
  const size_t nvec = size_t(n - head) / 2;
  const uint32_t tail = head + uint32_t(nvec * 2);
  if (blockIdx.x == gridDim.x - 1 && tid == 0) {
    if (head) count(a.keys64[0].x, a.keys64[0].y);
    if (tail < n) count(a.keys64[tail].x, a.keys64[tail].y);
  }
  const uint4* v4 = reinterpret_cast<const uint4*>(a.keys64 + head);
  size_t i = size_t(blockIdx.x) * kHist64Threads + tid;
  for (; i + 3 * stride < nvec; i += 4 * stride) {
    const uint4 x0 = ld_stream4(v4 + i);
    const uint4 x1 = ld_stream4(v4 + i + stride);
    const uint4 x2 = ld_stream4(v4 + i + 2 * stride);
    const uint4 x3 = ld_stream4(v4 + i + 3 * stride);
    count(x0.x, x0.y); count(x0.z, x0.w);
    count(x1.x, x1.y); count(x1.z, x1.w);
    count(x2.x, x2.y); count(x2.z, x2.w);
    count(x3.x, x3.y); count(x3.z, x3.w);
  }
  for (; i < nvec; i += stride) {
    const uint4 x = ld_stream4(v4 + i);
    count(x.x, x.y); count(x.z, x.w);
  }
  for (size_t z = size_t(blockIdx.x) * kHist64Threads + tid; z < a.zero_vec4; z += stride)
    a.zero_ptr[z] = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();
  // one row of 16 copies per (digit, bin)
  for (int r = tid; r < 8 * 256; r += kHist64Threads) {
    uint32_t sum = 0;
#pragma unroll
    for (int k = 0; k < 16; ++k) sum += sh[r * 16 + ((k + lane) & 15)];
    if (sum) atomicAdd(&a.hist[r], sum);
  }
}

cudaError_t launch_hist64(const HistArgs& a, unsigned grid, cudaStream_t s) {
  upfront_hist64_kernel<<<grid, kHist64Threads, kHist64Smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t prepare_hist64() {
  return cudaFuncSetAttribute(reinterpret_cast<const void*>(&upfront_hist64_kernel),
                              cudaFuncAttributeMaxDynamicSharedMemorySize, int(kHist64Smem));
}

// One block per digit: exclusive scan of its histogram, and whether a single
// bucket holds every key.
template <int R>
__global__ void __launch_bounds__((1 << R) < 1024 ? (1 << R) : 1024) digit_scan_kernel(const ScanArgs a) {
  constexpr int DIGITS = 1 << R;
  constexpr int THREADS = DIGITS < 1024 ? DIGITS : 1024;
  constexpr int PER = DIGITS / THREADS;
  __shared__ uint32_t s_warp[32];
  const int j = blockIdx.x, tid = threadIdx.x;
  const uint32_t* h = a.hist + size_t(j) * DIGITS + tid * PER;
  uint32_t v[PER], sum = 0;
  int full = 0;
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    v[k] = h[k];
    sum += v[k];
    full |= (v[k] == a.n);
  }
  uint32_t e = block_exclusive_sum<THREADS>(sum, s_warp);
  uint32_t* b = a.bases + size_t(j) * DIGITS + tid * PER;
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    b[k] = e;
    e += v[k];
  }
  const int any = __syncthreads_or(full);
  if (tid == 0 && a.skip) a.skip[j] = any ? 1u : 0u;
}

template <int R, int THREADS, int COPIES>
static cudaError_t launch_hist(const HistArgs& a, unsigned grid, cudaStream_t s) {
  const size_t smem = size_t(COPIES) * a.num_digits * (1u << R) * 4;
  if (is_identity(a.xform)) upfront_hist_kernel<R, THREADS, COPIES, false><<<grid, THREADS, smem, s>>>(a);
  else upfront_hist_kernel<R, THREADS, COPIES, true><<<grid, THREADS, smem, s>>>(a);
  return cudaGetLastError();
}

template <int R>
static cudaError_t launch_scan(const ScanArgs& a, unsigned grid, cudaStream_t s) {
  constexpr int THREADS = (1 << R) < 1024 ? (1 << R) : 1024;
  digit_scan_kernel<R><<<grid, THREADS, 0, s>>>(a);
  return cudaGetLastError();
}

// The four digits are the key's bytes, lowest first.
static bool byte_digits(const HistArgs& a) {
  if (a.num_digits != 4) return false;
  for (int j = 0; j < 4; ++j)
    if (a.dig[j].shift != uint32_t(8 * j) || a.dig[j].width != 8u) return false;
  return true;
}

template <int THREADS>
static cudaError_t launch_hist_lanes(const HistArgs& a, unsigned grid, cudaStream_t s) {
  const size_t smem = size_t(a.num_digits) * 256 * 32 * 4;
  if (byte_digits(a)) {
    if (is_identity(a.xform)) upfront_hist_lanes_kernel<THREADS, false, true><<<grid, THREADS, smem, s>>>(a);
    else upfront_hist_lanes_kernel<THREADS, true, true><<<grid, THREADS, smem, s>>>(a);
  } else {
    if (is_identity(a.xform)) upfront_hist_lanes_kernel<THREADS, false, false><<<grid, THREADS, smem, s>>>(a);
    else upfront_hist_lanes_kernel<THREADS, true, false><<<grid, THREADS, smem, s>>>(a);
  }
  return cudaGetLastError();
}

// Shared memory: 11-bit digits, 3 digits, 2 copies = 48 KiB; 8-bit digits,
// 4 digits x 256 bins x 32 lane copies = 128 KiB (one block per SM).
static const HistKernel kHist11 = {11, 512, size_t(2) * 3 * 2048 * 4, &launch_hist<11, 512, 2>,
                                   {reinterpret_cast<const void*>(&upfront_hist_kernel<11, 512, 2, false>),
                                    reinterpret_cast<const void*>(&upfront_hist_kernel<11, 512, 2, true>)}};
static const HistKernel kHist8 = {8, 1024, size_t(4) * 256 * 32 * 4, &launch_hist_lanes<1024>,
                                  {reinterpret_cast<const void*>(&upfront_hist_lanes_kernel<1024, false, false>),
                                   reinterpret_cast<const void*>(&upfront_hist_lanes_kernel<1024, true, false>),
                                   reinterpret_cast<const void*>(&upfront_hist_lanes_kernel<1024, false, true>),
                                   reinterpret_cast<const void*>(&upfront_hist_lanes_kernel<1024, true, true>)}};
static const ScanKernel kScan11 = {11, 1024, &launch_scan<11>};
static const ScanKernel kScan8 = {8, 256, &launch_scan<8>};

const HistKernel* hist_kernel(int radix_bits) { return radix_bits == 11 ? &kHist11 : (radix_bits == 8 ? &kHist8 : nullptr); }
const ScanKernel* scan_kernel(int radix_bits) { return radix_bits == 11 ? &kScan11 : (radix_bits == 8 ? &kScan8 : nullptr); }

}  // namespace rs
