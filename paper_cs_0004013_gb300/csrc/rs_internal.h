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

// Order-preserving map of a 32-bit key word onto an unsigned one, so that
// signed and IEEE-754 binary32 keys sort by the same unsigned radix passes
// (the paper sorts positive integers, Sec. 1.1):
//   ordered = key ^ ((sign(key) ? fmask : 0) ^ smask)
// unsigned: (0, 0); two's-complement signed: (0, 0x80000000), the sign bit
// flipped; binary32: (0x7fffffff, 0x80000000), every bit of a negative value
// flipped and the sign bit of a non-negative one (the total order
// -NaN < -inf < ... < -0 < +0 < ... < +inf < +NaN of IEEE 754 totalOrder).
struct KeyXform {
  uint32_t fmask, smask;
};
constexpr KeyXform kIdentityXform = {0u, 0u};

// The same map for 64-bit keys held as (low word, high word): the sign is
// the high word's top bit; a set sign flips the low word by flo and the high
// word by fhi, and shi is flipped in the high word of every key.
// unsigned: (0, 0, 0); signed: (0, 0, 0x80000000); binary64:
// (0xffffffff, 0x7fffffff, 0x80000000).
struct KeyXform64 {
  uint32_t flo, fhi, shi;
};

// Split of interleaved 64-bit keys into word planes, and the join back.
struct WideArgs {
  const uint2* keys;  // split: the input keys
  uint2* out;         // join: the output keys
  uint32_t* lo;       // [n] low words
  uint32_t* hi;       // [n] high words
  uint64_t n;
  KeyXform64 x;
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
  KeyXform xform;      // applied to every key before its digits are taken
  // launch_hist64 only: interleaved 64-bit keys and their order map
  const uint2* keys64;
  KeyXform64 x64;
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
  const uint32_t* vals2_in;  // a second payload word (kernels with two)
  uint32_t* vals2_out;
  uint32_t* vals2_alt;
  uint32_t n;
  uint32_t shift, width;
  int pass, num_passes;
  const uint32_t* bases;     // [2^R] of this pass's digit
  const uint32_t* skip;      // [num_passes] or null
  void* status;              // [num_tiles][2^R] status words
  uint32_t* tile_counter;    // this pass's tile ticket, zeroed before the launch
  uint32_t* err;             // device error word
  KeyXform xin;              // applied to keys read from keys_in
  KeyXform xout;             // inverted on keys written to keys_out
  // Interleaved two-word elements in place of two word planes (non-persistent
  // kernels with payload words only).  The first executed pass reads them from
  // pair_in, the last one writes them to pair_out; either may be null.
  // pair_key = 1: 64-bit keys (order map x64); word key_high (0 low, 1 high)
  // is this pass's key and the other word is payload word 1.  pair_key = 0:
  // 64-bit values, payload words 1 and 2.
  const uint2* pair_in;
  uint2* pair_out;
  int pair_key;
  uint32_t key_high;
  KeyXform64 x64;
  // Values sorted through an index (non-persistent kernels with two payload
  // words): with iota the first executed pass makes the last payload word the
  // element's input index; with gather_out the last executed pass writes
  // gather[index] (n elements) to gather_out in its place.
  int iota;
  const uint2* gather;
  uint2* gather_out;
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
  int persistent_per_sm = 0;  // > 0: persistent kernel, grid = SMs x this (capped by tiles)
  int value_words = -1;       // payload words per key (-1: 1 if pairs else 0)
  bool pair_io = false;       // reads and writes interleaved 64-bit words (PassArgs pair_* and gather fields)
  // Keys only: the kernel for pass 0, which ranks without keeping the order of
  // equal digits when it is the sort's first executed pass (null: `launch`).
  cudaError_t (*launch_first)(const PassArgs&, unsigned grid, cudaStream_t) = nullptr;
  const void* func_first = nullptr;
  int vwords() const { return value_words >= 0 ? value_words : (pairs ? 1 : 0); }
};

struct HistKernel {
  int radix_bits;
  int threads;
  size_t smem;
  cudaError_t (*launch)(const HistArgs&, unsigned grid, cudaStream_t);
  const void* funcs[4];  // every instance (for attributes); unused entries null
};

struct ScanKernel {
  int radix_bits;
  int threads;
  cudaError_t (*launch)(const ScanArgs&, unsigned grid, cudaStream_t);
};

// ---- segmented pipeline (segmented.cu) ---------------------------------------
// Words of the device counts array written by seg_plan.
enum : int { SEG_NUM_LARGE = 0, SEG_NUM_SMALL = 1, SEG_NUM_TINY = 2, SEG_NUM_TILES = 3, SEG_TICKETS = 4 };
// counts[SEG_TICKETS + p] is the tile ticket of pass p; the array has
// SEG_TICKETS + kMaxDigits words.
constexpr int kSegCountWords = SEG_TICKETS + kMaxDigits;

struct SegPlanArgs {
  const uint64_t* seg_off;  // [num_segs + 1]
  uint32_t num_segs;
  uint32_t tiny_max, small_max, tile;
  uint32_t* large_seg;      // [num_segs] ids of large segments
  uint32_t* tile_prefix;    // [num_segs + 1] first tile of each large segment
  uint32_t* small_seg;      // [num_segs]
  uint32_t* tiny_seg;       // [num_segs]
  uint32_t* counts;         // [kSegCountWords]
};

// Where one tile of a large segment lies (written by seg_hist, read by
// every seg_pass launch so that a tile costs one lookup).
struct SegTileJob {
  uint64_t base;       // index of the tile's first key
  uint32_t valid;      // keys in the tile
  uint32_t first;      // first tile of the segment
  uint32_t out_start;  // segment start and end in the output
  uint32_t out_end;
  uint32_t li;         // index of the segment among the large ones
  uint32_t reserved;
};
static_assert(sizeof(SegTileJob) == 32, "two 16-byte words per tile");

struct SegHistArgs {
  const uint32_t* keys;
  const uint64_t* seg_off;
  const uint32_t* large_seg;
  const uint32_t* tile_prefix;
  const uint32_t* counts;
  uint32_t tile;
  int num_digits;
  DigitSpec dig[kMaxDigits];
  uint32_t* seg_hist;  // [num_large][num_digits][256], zeroed before the launch
  uint32_t* status;    // [tiles][256]; each tile's row is cleared here
  SegTileJob* jobs;    // [tiles]; written here
  KeyXform xform;      // applied to every key before its digits are taken
};

struct SegScanArgs {
  const uint32_t* seg_hist;
  uint32_t* seg_bases;  // same shape
  const uint32_t* counts;
  int num_digits;
};

struct SegPassArgs {
  const uint32_t* kin;
  uint32_t* kout;
  const uint32_t* vin;
  uint32_t* vout;
  const uint32_t* counts;
  const uint32_t* seg_bases;
  const SegTileJob* jobs;
  int num_digits, pass;
  uint32_t shift, width;
  uint32_t* status;
  uint32_t* tile_counter;
  uint32_t parity;
  uint32_t* err;
  KeyXform xin, xout;  // applied on loading kin, inverted on storing kout
};

struct LocalArgs {
  const uint32_t* kin;
  uint32_t* kout;
  const uint32_t* vin;
  uint32_t* vout;
  const uint64_t* seg_off;
  const uint32_t* list;   // segment ids (null: one array of single_n keys)
  const uint32_t* count;  // device count of list entries
  uint32_t single_n;      // keys of the one array when list is null (<= the block's tile)
  int num_digits;
  DigitSpec dig[kMaxDigits];
  KeyXform xin, xout;     // applied on loading kin, inverted on storing kout
};

// Tiled-pass shapes of the segmented pipeline (rs_plan.tile = shape + 1).
constexpr int kSegShapes = 3;

struct SegKernels {
  uint32_t tile_keys[kSegShapes], tile_pairs[kSegShapes], tiny_max, small_max;
  uint32_t blocks_per_sm[kSegShapes];  // the persistent pass's resident blocks
  uint32_t tile(bool pairs, int shape) const { return pairs ? tile_pairs[shape] : tile_keys[shape]; }
  size_t pass_smem_keys[kSegShapes], pass_smem_pairs[kSegShapes];
  size_t tiny_smem_keys, tiny_smem_pairs, small_smem_keys, small_smem_pairs;
  const void* pass_keys[kSegShapes];
  const void* pass_pairs[kSegShapes];
  const void* tiny_keys;
  const void* tiny_pairs;
  const void* small_keys;
  const void* small_pairs;
  const void* hist;     // the segment histogram kernel for unsigned keys
  const void* hist_xf;  // and for keys of another kind
  size_t hist_smem;
};

const SegKernels* seg_kernels();
cudaError_t launch_seg_plan(const SegPlanArgs& a, cudaStream_t s);
cudaError_t launch_seg_hist(const SegHistArgs& a, unsigned grid, cudaStream_t s);
cudaError_t launch_seg_scan(const SegScanArgs& a, unsigned grid, cudaStream_t s);
cudaError_t launch_seg_pass(const SegPassArgs& a, bool pairs, int shape, unsigned grid, cudaStream_t s);
cudaError_t launch_local_sort(const LocalArgs& a, bool small, bool pairs, unsigned grid, cudaStream_t s);
cudaError_t launch_bases_to_offsets(const uint32_t* bases, uint32_t num, uint64_t n, uint64_t* seg_off,
                                    cudaStream_t s);

// Stable merge of two sorted runs (merge.cu).
struct MergeArgs {
  const uint32_t* a;   // [na] sorted by the order of x
  const uint32_t* b;   // [nb] sorted by the order of x
  const uint32_t* va;  // payloads of a, b (both null for keys only)
  const uint32_t* vb;
  uint32_t* out;       // [na + nb]
  uint32_t* vout;
  uint32_t na, nb;
  uint32_t* split;     // [tiles + 1] merge-path split of each tile boundary
  KeyXform x;
  uint32_t* err;       // device error word
  uint32_t tile;       // outputs per tile (merge_tile_keys of the chosen shape)
};
uint32_t merge_tile_keys(uint32_t shape, bool pairs);
cudaError_t launch_merge(const MergeArgs& m, cudaStream_t s);

cudaError_t launch_split64(const WideArgs& a, unsigned grid, cudaStream_t s);
cudaError_t launch_join64(const WideArgs& a, unsigned grid, cudaStream_t s);

// A whole sort of up to a few million keys in one cooperative launch
// (fused.cu): 8-bit digits, one 384 x 24, 384 x 18 or 384 x 12 tile per block, every block resident.
struct FusedArgs {
  const uint32_t* keys_in;
  uint32_t* keys_out;
  uint32_t* keys_alt;
  const uint32_t* vals_in;   // null for keys only
  uint32_t* vals_out;
  uint32_t* vals_alt;
  uint32_t n;
  KeyXform xf;               // order map of the keys' kind
  uint32_t* hist;            // [4][256], zero on entry
  void* status;              // [tiles][256] 32-bit status words, zero on entry
  uint32_t* bar;             // barrier counter, zero on entry
  uint32_t* err;             // device error word
};
constexpr int kFusedShapes = 3;  // tile shapes of the single-launch sort: 384 x 24, 384 x 18, 384 x 12
uint32_t fused_tile_keys(int shape);
size_t fused_smem(bool pairs, int shape);
const void* fused_func(bool pairs, int shape);
cudaError_t launch_fused(const FusedArgs& a, unsigned tiles, bool pairs, int shape, cudaStream_t s);

// The MSD plan's bucketing (msd.cu): bucket = order-mapped key >> kMsdShift
// (2^14 buckets); C chunks of ceil(n / C) keys, one block each.
constexpr uint32_t kMsdShift = 18;
struct MsdArgs {
  const uint32_t* keys;
  uint64_t n;
  KeyXform x;
  uint32_t chunks;
  uint32_t* hist;     // [chunks][2^14]: counts, then exclusive down each bucket's column
  uint32_t* totals;   // [2^14]: bucket totals, then bucket bases
  uint64_t* seg_off;  // [2^14 + 1]: bucket bases as segment offsets (last = n)
  uint32_t* out;      // [n] bucketed, order-mapped keys (keys-only distribution)
  uint32_t* err;      // device error word
};
size_t msd_smem();
const void* msd_count_func();
const void* msd_scatter_func();
cudaError_t launch_msd_count(const MsdArgs& a, cudaStream_t s);
cudaError_t launch_msd_scan(const MsdArgs& a, cudaStream_t s);
cudaError_t launch_msd_scatter(const MsdArgs& a, cudaStream_t s);

// The selection of Sec. 4.2.1 (select.cu): an evenly spaced sample of at
// most 1024 keys, bucketed by the top `bits` of its significant width;
// out[0] = problem cells, out[1] = 1 if more than max_problem, out[2] = the
// bucket shift, out[3] = the sample size; buckets (may be null) receives the
// sorted sample buckets.
struct SelectArgs {
  const uint32_t* keys;
  uint64_t n;
  KeyXform x;
  uint32_t bits, sample, cells, max_problem;
  uint32_t* out;      // [4], device
  uint32_t* buckets;  // [sample] or null, device
};
cudaError_t launch_select(const SelectArgs& a, cudaStream_t s);

// Self-test of the bounded lookback wait (selftest.cu).
cudaError_t launch_lookback_timeout(const uint32_t* status, uint32_t* err, cudaStream_t s);

// Sets the calling thread's message for rs_last_error() (printf format).
void set_last_error(int status, const char* fmt, ...);

// Registries (defined in the kernel translation units).
const OnesweepKernel* onesweep_kernels_r8(int* count);
const OnesweepKernel* onesweep_kernels_r11(int* count);
const HistKernel* hist_kernel(int radix_bits);
// All eight byte-digit histograms of interleaved 64-bit keys (HistArgs keys64,
// x64; hist is [8][256]) in one read; prepare_hist64 sets its shared-memory size.
cudaError_t launch_hist64(const HistArgs& a, unsigned grid, cudaStream_t s);
cudaError_t prepare_hist64();
const ScanKernel* scan_kernel(int radix_bits);

}  // namespace rs
