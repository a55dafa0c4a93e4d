// Internal interface between the C-ABI layer (api.cu) and the kernels.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace rs {

constexpr int kMaxDigits = 4;  // digits of a plan over 32-bit keys (8-bit digits)

struct DigitSpec {
  uint32_t shift, width;
};

// Upfront histogram (one read of the keys, every digit at once) and zeroing
// of the chained-scan status array.
struct HistArgs {
  const uint32_t* keys;
  uint32_t n;
  int num_digits;
  DigitSpec dig[kMaxDigits];
  uint32_t* hist;      // [num_digits][2^R], zeroed before the launch
  uint4* zero_ptr;     // region to clear (status words), may be null
  size_t zero_vec4;    // its size in 16-byte units
};

// Exclusive scan of each digit's histogram + skip flags.
struct ScanArgs {
  const uint32_t* hist;  // [num_digits][2^R]
  uint32_t* bases;       // [num_digits][2^R]
  uint32_t* skip;        // [num_digits] (may be null)
  uint32_t n;
};

// One onesweep LSD pass.
struct PassArgs {
  const uint32_t* keys_in;
  uint32_t* keys_out;
  uint32_t* keys_alt;
  const uint32_t* vals_in;
  uint32_t* vals_out;
  uint32_t* vals_alt;
  uint32_t n;
  uint32_t shift, width;
  int pass, num_passes;
  const uint32_t* bases;     // [2^R] of this pass's digit
  const uint32_t* skip;      // [num_passes] or null
  void* status;              // [num_tiles][2^R] status words
  uint32_t* tile_counter;    // this pass's tile ticket, zeroed before the launch
  uint32_t* err;             // device error word
};

struct OnesweepKernel {
  int radix_bits;
  int shape;         // tile-shape index (0 = default) selected by rs_plan.tile - 1
  int threads;
  int items;
  int tile;          // keys per tile
  bool pairs;
  bool wide_status;  // 64-bit status words (n >= 2^30)
  size_t smem;       // dynamic shared memory bytes
  cudaError_t (*launch)(const PassArgs&, unsigned grid, cudaStream_t);
  const void* func;  // kernel symbol (for attributes)
};

struct HistKernel {
  int radix_bits;
  int threads;
  size_t smem;
  cudaError_t (*launch)(const HistArgs&, unsigned grid, cudaStream_t);
  const void* func;
};

struct ScanKernel {
  int radix_bits;
  int threads;
  cudaError_t (*launch)(const ScanArgs&, unsigned grid, cudaStream_t);
};

// Sets the calling thread's message for rs_last_error() (printf format).
void set_last_error(int status, const char* fmt, ...);

// Registries (defined in the kernel translation units).
const OnesweepKernel* onesweep_kernels_r8(int* count);
const OnesweepKernel* onesweep_kernels_r11(int* count);
const HistKernel* hist_kernel(int radix_bits);
const ScanKernel* scan_kernel(int radix_bits);

}  // namespace rs
