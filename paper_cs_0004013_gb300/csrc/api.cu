// C ABI of librsort (declared in include/rsort.h): argument checks, the
// radix plan, the layout of the caller's temp buffer and the launches.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "rs_device.cuh"
#include "rs_internal.h"
#include "rsort.h"

namespace rs {
namespace {

constexpr uint32_t kVersion = 1 * 10000 + 0 * 100 + 0;
constexpr int kMaxDevices = 64;
constexpr size_t kAlign = 256;

thread_local std::string g_last_error;

rs_status fail(rs_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

rs_status cuda_fail(cudaError_t e, const char* what) {
  return fail(RS_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

#define RS_CUDA(call, what)                   \
  do {                                        \
    cudaError_t e_ = (call);                  \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

// Device error word: set by kernels whose bounded waits gave up.
__device__ uint32_t g_err_word;
// Where the selection kernel leaves its four result words (read back by the host).
__device__ uint32_t g_select_out[4];
std::mutex g_select_mu;  // one selection at a time per process (they share the result words)
// Where take_error_kernel leaves the word it took (read back by the host).
__device__ uint32_t g_err_taken;

// Reads and clears the error word in one atomic step, so that a bit a kernel
// on another stream sets in between is kept for the next check, not lost.
__global__ void take_error_kernel(uint32_t* err, uint32_t* taken) { *taken = atomicExch(err, 0u); }

struct DeviceState {
  bool ready = false;
  uint32_t* err = nullptr;
  uint32_t* err_taken = nullptr;
  int num_sms = 0;
  uint32_t fused_tiles[2][kFusedShapes] = {};  // tiles the single-launch sort holds resident ([pairs][shape])
};
std::mutex g_mu;
std::mutex g_err_mu;  // one error-word check at a time (they share the copy word)
DeviceState g_dev[kMaxDevices];

rs_status device_state(DeviceState** out) {
  int dev = 0;
  RS_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return fail(RS_ERR_UNSUPPORTED, "device index %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_mu);
  DeviceState& st = g_dev[dev];
  if (!st.ready) {
    RS_CUDA(cudaGetSymbolAddress(reinterpret_cast<void**>(&st.err), g_err_word), "cudaGetSymbolAddress(error word)");
    RS_CUDA(cudaGetSymbolAddress(reinterpret_cast<void**>(&st.err_taken), g_err_taken),
            "cudaGetSymbolAddress(error word copy)");
    RS_CUDA(cudaDeviceGetAttribute(&st.num_sms, cudaDevAttrMultiProcessorCount, dev), "cudaDeviceGetAttribute");
    int cnt = 0;
    for (int r : {8, 11}) {
      const OnesweepKernel* ks = r == 8 ? onesweep_kernels_r8(&cnt) : onesweep_kernels_r11(&cnt);
      for (int i = 0; i < cnt; ++i) {
        RS_CUDA(cudaFuncSetAttribute(ks[i].func, cudaFuncAttributeMaxDynamicSharedMemorySize, int(ks[i].smem)),
                "cudaFuncSetAttribute(onesweep)");
        if (ks[i].func_first)
          RS_CUDA(cudaFuncSetAttribute(ks[i].func_first, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       int(ks[i].smem)),
                  "cudaFuncSetAttribute(onesweep first pass)");
      }
      const HistKernel* h = hist_kernel(r);
      for (const void* f : h->funcs)
        if (f)
          RS_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, int(h->smem)),
                  "cudaFuncSetAttribute(hist)");
    }
    RS_CUDA(prepare_hist64(), "cudaFuncSetAttribute(hist64)");
    for (const void* f : {msd_count_func(), msd_scatter_func()})
      RS_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, int(msd_smem())),
              "cudaFuncSetAttribute(msd)");
    int coop = 0;
    RS_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev), "cudaDeviceGetAttribute(coop)");
    for (int pr = 0; pr < 2; ++pr)
      for (int sh = 0; sh < kFusedShapes; ++sh) {
        RS_CUDA(cudaFuncSetAttribute(fused_func(pr != 0, sh), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     int(fused_smem(pr != 0, sh))),
                "cudaFuncSetAttribute(fused)");
        int per_sm = 0;
        RS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fused_func(pr != 0, sh), 384,
                                                              fused_smem(pr != 0, sh)),
                "cudaOccupancyMaxActiveBlocksPerMultiprocessor(fused)");
        st.fused_tiles[pr][sh] = coop ? uint32_t(per_sm) * uint32_t(st.num_sms) : 0u;
      }
    const SegKernels* sk = seg_kernels();
    const void* fn[12] = {sk->pass_keys[0], sk->pass_pairs[0], sk->pass_keys[1], sk->pass_pairs[1],
                          sk->pass_keys[2], sk->pass_pairs[2], sk->tiny_keys,    sk->tiny_pairs,
                          sk->small_keys,   sk->small_pairs,   sk->hist,         sk->hist_xf};
    const size_t sm[12] = {sk->pass_smem_keys[0], sk->pass_smem_pairs[0], sk->pass_smem_keys[1],
                           sk->pass_smem_pairs[1], sk->pass_smem_keys[2],  sk->pass_smem_pairs[2],
                           sk->tiny_smem_keys,     sk->tiny_smem_pairs,    sk->small_smem_keys,
                           sk->small_smem_pairs,   sk->hist_smem,          sk->hist_smem};
    for (int i = 0; i < 12; ++i)
      RS_CUDA(cudaFuncSetAttribute(fn[i], cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm[i])),
              "cudaFuncSetAttribute(segmented)");
    st.ready = true;
  }
  *out = &st;
  return RS_OK;
}

// ---- tracing -------------------------------------------------------------------
enum TraceKind {
  T_CLEAR = 0, T_HIST, T_SCAN, T_PASS8, T_PASS11, T_SEGOFF, T_SEGPLAN, T_SEGHIST, T_SEGSCAN, T_SEGPASS, T_LOCAL,
  T_H2D, T_D2H, T_SPLIT, T_JOIN, T_MERGE, T_SELECT, T_MSDCOUNT, T_MSDSCAN, T_MSDSCATTER, T_FUSED, T_KINDS
};
const char* const kTraceNames[T_KINDS] = {"clear",       "upfront_hist", "digit_scan", "onesweep_r8",
                                          "onesweep_r11", "seg_part_offsets", "seg_plan", "seg_hist",
                                          "seg_scan",    "seg_pass",     "local_sort", "copy_h2d",
                                          "copy_d2h",    "split64",      "join64",     "merge",
                                          "select",      "msd_count",    "msd_scan",   "msd_scatter",
                                          "fused_sort"};

// The selection of Sec. 4.2.1 with the paper's parameters: a 1000-point
// sample (footnote 8), 64 cells, 65 % overlap, more than two problem cells;
// buckets of the top 13 significant bits (the paper's 8192 buckets, Sec. 4.7).
constexpr uint32_t kSelectSample = 1000, kSelectCells = 64, kSelectMaxProblem = 2, kSelectBits = 13;
struct TraceRec {
  int kind;
  double keys;
  cudaEvent_t a, b;
};
std::mutex g_trace_mu;
bool g_trace_on = false;
std::vector<TraceRec> g_trace;
std::vector<cudaEvent_t> g_event_pool;

cudaError_t take_event(cudaEvent_t* e) {
  if (!g_event_pool.empty()) {
    *e = g_event_pool.back();
    g_event_pool.pop_back();
    return cudaSuccess;
  }
  return cudaEventCreate(e);
}

// Runs `launch` (which enqueues one kernel or memset on s), bracketed by
// events when tracing is on.
template <class F>
cudaError_t traced(int kind, double keys, cudaStream_t s, F&& launch) {
  std::unique_lock<std::mutex> lock(g_trace_mu);
  if (!g_trace_on) {
    lock.unlock();
    return launch();
  }
  TraceRec r{kind, keys, nullptr, nullptr};
  cudaError_t e = take_event(&r.a);
  if (e == cudaSuccess) e = take_event(&r.b);
  if (e == cudaSuccess) e = cudaEventRecord(r.a, s);
  if (e != cudaSuccess) return e;
  e = launch();
  if (e != cudaSuccess) return e;
  e = cudaEventRecord(r.b, s);
  if (e == cudaSuccess) g_trace.push_back(r);
  return e;
}

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
  if (!a || !b || na == 0 || nb == 0) return false;
  const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  return x < y + nb && y < x + na;
}

// ---- default plans per entry point and size class ----------------------------
// A tuner (or the caller) may install the plan an entry point uses for a size
// class when the caller passes no plan or leaves fields zero.  Size class =
// ceil(log2(n)) for plain sorts, ceil(log2(mean segment size)) for segmented
// ones.  Unset classes keep the compiled defaults.
constexpr int kPlanEntries = 4;
constexpr int kSizeClasses = 33;
std::mutex g_plan_mu;
rs_plan g_plan_table[kPlanEntries][kSizeClasses] = {};
bool g_plan_set[kPlanEntries][kSizeClasses] = {};

uint32_t size_log2(uint64_t n) {
  uint32_t b = 0;
  while (b < 32 && (uint64_t(1) << b) < n) ++b;
  return b;
}

// The plan an entry point runs: the caller's nonzero fields, else the
// installed plan's, else zero (the compiled defaults).  key_kind is always
// the caller's (zero, unsigned, without a plan).
rs_plan resolve_plan(int entry, uint64_t size, const rs_plan* user) {
  rs_plan r = {0, 0, 0, 0};
  {
    std::lock_guard<std::mutex> lock(g_plan_mu);
    const uint32_t c = size_log2(size);
    if (g_plan_set[entry][c]) r = g_plan_table[entry][c];
  }
  r.key_kind = 0;
  if (user) {
    if (user->digit_bits) r.digit_bits = user->digit_bits;
    if (user->mode) r.mode = user->mode;
    if (user->tile) r.tile = user->tile;
    r.key_kind = user->key_kind;
  }
  return r;
}

// ---- plan -------------------------------------------------------------------
struct SortPlan {
  KeyXform xf = kIdentityXform;  // order map of the plan's key kind
  int R = 11;
  bool msd = false;  // top-digit bucketing pass, then the segmented pipeline per bucket
  int nd = 0;
  DigitSpec dig[kMaxDigits] = {};
  const OnesweepKernel* k = nullptr;
  size_t num_tiles = 0;
  size_t status_rows = 0;  // status rows to hold when more than num_tiles (the single-launch sort's small tiles)
};

// Defaults from measurement on GB300 (uniform 31-bit keys, 2^16 .. 2^26):
// 8-bit digits beat 11-bit ones (four 8-bit passes take less time than
// three 11-bit ones); LSD beats the MSD plan at every size (the MSD plan's
// distribution and local sorts cost more SM work than the passes it saves).
int default_digit_bits(uint64_t /*n*/, bool /*pairs*/) { return 8; }
uint32_t default_mode(uint64_t /*n*/, bool /*pairs*/) { return RS_MODE_LSD; }
// Tiles of the 8-bit passes (explicit LSD plans; the automatic plan sorts up
// to a few million keys in one launch): keys take the half-warp-group kernel
// at 384 x 24 at every size (2^20 keys: 93.5 us per sort against 95.2 for
// the lane-mask kernel at 512 x 16; 2^22: 134 against 156; 2^26: 0.98 ms
// against 1.12 at 512 x 24); key+payload sorts the lane-mask kernel at
// 512 x 16 up to 2^21 keys (2^21: 120 us against 123 at 384 x 24 and 131 at
// 512 x 24) and at 384 x 24, three blocks per SM, above (2^22: 159 us against
// 172 and 174; 2^26: 322 us per pass against 332 at 512 x 24 and 362 for the
// half-warp-group kernel, which loads the payloads after ranking).
uint32_t default_tile(int R, bool pairs, uint64_t n) {
  if (R == 8) return pairs ? (n <= (uint64_t(1) << 21) ? 1u : 8u) : 2u;
  return pairs ? 1u : 4u;
}

// n + one tile must fit the 30-bit count field of 32-bit status words.
bool needs_wide_status(uint64_t n) { return n + 65536 > uint64_t(StatusCodec<uint32_t>::kVal); }

rs_status pick_kernel(int R, uint32_t tile_idx, int vwords, bool wide, const OnesweepKernel** out) {
  int cnt = 0;
  const OnesweepKernel* ks = R == 8 ? onesweep_kernels_r8(&cnt) : onesweep_kernels_r11(&cnt);
  const int shape = tile_idx == 0 ? 0 : int(tile_idx) - 1;
  const bool pairs = vwords > 0;
  bool any = false, any_payload = false;
  for (int i = 0; i < cnt; ++i) {
    if (ks[i].shape != shape) continue;
    any = true;
    any_payload |= ks[i].vwords() == vwords;
    if (ks[i].vwords() == vwords && ks[i].wide_status == wide) {
      *out = &ks[i];
      return RS_OK;
    }
  }
  if (!any) return fail(RS_ERR_UNSUPPORTED, "tile shape %u not available for %d-bit digits", tile_idx, R);
  if (!any_payload)
    return fail(RS_ERR_UNSUPPORTED, "tile shape %u has no kernel moving %d payload word(s)", tile_idx, vwords);
  (void)pairs;
  return fail(RS_ERR_UNSUPPORTED, "tile shape %u has no %s-status kernel (n too large for it)", tile_idx,
              wide ? "64-bit" : "32-bit");
}

// The variant of a pass kernel that reads and writes interleaved 64-bit
// words (same shape, payload words and status width), or null.
const OnesweepKernel* pair_io_kernel(const OnesweepKernel* k) {
  if (k->pair_io) return k;
  int cnt = 0;
  const OnesweepKernel* ks = k->radix_bits == 8 ? onesweep_kernels_r8(&cnt) : onesweep_kernels_r11(&cnt);
  for (int i = 0; i < cnt; ++i)
    if (ks[i].pair_io && ks[i].shape == k->shape && ks[i].vwords() == k->vwords() &&
        ks[i].wide_status == k->wide_status)
      return &ks[i];
  return nullptr;
}

// The order map of a key kind (see KeyXform).
rs_status key_xform(const rs_plan* user, KeyXform* out) {
  const uint32_t kind = user ? user->key_kind : uint32_t(RS_KEY_U32);
  switch (kind) {
    case RS_KEY_U32: *out = KeyXform{0u, 0u}; return RS_OK;
    case RS_KEY_I32: *out = KeyXform{0u, 0x80000000u}; return RS_OK;
    case RS_KEY_F32: *out = KeyXform{0x7fffffffu, 0x80000000u}; return RS_OK;
    default: return fail(RS_ERR_INVALID, "unknown key_kind %u", kind);
  }
}

// vwords: payload words per key the passes move (-1: 1 for pairs, else 0).
rs_status make_plan(uint64_t n, bool pairs, const rs_plan* user, SortPlan* p, int vwords = -1) {
  if (rs_status st = key_xform(user, &p->xf); st != RS_OK) return st;
  const uint32_t bits = (user && user->digit_bits) ? user->digit_bits : uint32_t(default_digit_bits(n, pairs));
  if (bits != 8 && bits != 11) return fail(RS_ERR_UNSUPPORTED, "digit_bits must be 8 or 11 (got %u)", bits);
  if (user && user->mode > RS_MODE_MSD) return fail(RS_ERR_INVALID, "unknown mode %u", user->mode);
  const uint32_t mode = (user && user->mode) ? user->mode : (bits == 8 ? default_mode(n, pairs) : RS_MODE_LSD);
  p->msd = mode == RS_MODE_MSD;
  if (p->msd && bits != 8) return fail(RS_ERR_UNSUPPORTED, "the MSD plan uses 8-bit digits");
  if (p->msd && needs_wide_status(n)) return fail(RS_ERR_UNSUPPORTED, "the MSD plan needs n < 2^30 - 2^16");
  p->R = int(bits);
  p->nd = 0;
  for (uint32_t s = 0; s < 32; s += bits) {
    p->dig[p->nd].shift = s;
    p->dig[p->nd].width = (32 - s) < bits ? (32 - s) : bits;
    ++p->nd;
  }
  const bool wide = needs_wide_status(n);
  uint32_t tile = (user && user->tile) ? user->tile : default_tile(p->R, pairs, n);
  // 64-bit status kernels: shapes 0, 1 and 4 (keys and pairs), shape 2 (keys)
  if (wide && !(user && user->tile)) tile = (pairs || p->R != 8) ? 1u : 2u;
  rs_status st = pick_kernel(p->R, tile, vwords >= 0 ? vwords : (pairs ? 1 : 0), wide, &p->k);
  if (st != RS_OK) return st;
  p->num_tiles = (n + p->k->tile - 1) / p->k->tile;
  return RS_OK;
}

// ---- temp layout ------------------------------------------------------------
struct Layout {
  size_t ctrl = 0;     // [0,16): tile tickets per pass; [16,32): skip flags
  size_t hist = 0;     // [nd][2^R] u32
  size_t bases = 0;    // [nd][2^R] u32
  size_t status = 0;   // [num_tiles][2^R] status words
  size_t status_bytes = 0;
  size_t alt_k = 0, alt_v = 0;
  size_t memset_bytes = 0;  // ctrl + hist, cleared before the histogram
  size_t total = 0;
};

Layout make_layout(const SortPlan& p, uint64_t n, bool pairs) {
  Layout L;
  const size_t digits = size_t(1) << p.R;
  size_t off = 0;
  L.ctrl = off;
  off += kAlign;
  L.hist = off;
  off = align_up(off + size_t(p.nd) * digits * 4);
  L.memset_bytes = off;
  L.bases = off;
  off = align_up(off + size_t(p.nd) * digits * 4);
  L.status = off;
  L.status_bytes = (p.status_rows > p.num_tiles ? p.status_rows : p.num_tiles) * digits * (p.k->wide_status ? 8 : 4);
  off = align_up(off + L.status_bytes);
  if (p.nd > 1 && n > 0) {
    L.alt_k = off;
    off = align_up(off + size_t(n) * 4);
    if (pairs) {
      L.alt_v = off;
      off = align_up(off + size_t(n) * 4);
    }
  }
  L.total = off;
  return L;
}

// Blocks of a pass launch: one per tile, or for persistent kernels as many
// as stay resident (capped by the tile count).
unsigned pass_grid(const SortPlan& p, const DeviceState* ds) {
  size_t g = p.num_tiles;
  if (p.k->persistent_per_sm > 0) {
    const size_t cap = size_t(ds->num_sms) * size_t(p.k->persistent_per_sm);
    if (cap < g) g = cap;
  }
  return unsigned(g > 0 ? g : 1);
}

void part_offsets_host(uint64_t n, uint32_t parts, uint64_t* out) {
  const uint64_t q = n / parts, r = n % parts;
  for (uint64_t p = 0; p <= parts; ++p) out[p] = p * q + (p < r ? p : r);
}

// ---- the LSD pipeline ---------------------------------------------------------
// memset(ctrl + hist) -> upfront histogram (+ clear status) -> digit scans ->
// one onesweep pass per digit.
// vals2_*: a second payload word per key (kernels with two payload words),
// its input, output and alternate planes; null for one word or none.
rs_status run_lsd(const SortPlan& p, const Layout& L, const uint32_t* keys_in, const uint32_t* vals_in,
                  uint32_t* keys_out, uint32_t* vals_out, uint32_t n, unsigned char* temp, bool force_all,
                  DeviceState* ds, cudaStream_t s, const uint32_t* vals2_in = nullptr, uint32_t* vals2_out = nullptr,
                  uint32_t* vals2_alt = nullptr, const uint2* pair_vals_in = nullptr, uint2* pair_vals_out = nullptr) {
  uint32_t* ctrl = reinterpret_cast<uint32_t*>(temp + L.ctrl);
  uint32_t* hist = reinterpret_cast<uint32_t*>(temp + L.hist);
  uint32_t* bases = reinterpret_cast<uint32_t*>(temp + L.bases);
  const size_t digits = size_t(1) << p.R;
  RS_CUDA(traced(T_CLEAR, 0, s, [&] { return cudaMemsetAsync(temp, 0, L.memset_bytes, s); }),
          "cudaMemsetAsync(temp)");

  HistArgs ha{};
  ha.keys = keys_in;
  ha.n = n;
  ha.num_digits = p.nd;
  for (int j = 0; j < p.nd; ++j) ha.dig[j] = p.dig[j];
  ha.hist = hist;
  ha.zero_ptr = reinterpret_cast<uint4*>(temp + L.status);
  ha.zero_vec4 = L.status_bytes / 16;
  ha.xform = p.xf;
  const HistKernel* hk = hist_kernel(p.R);
  const size_t work = (size_t(n) + 4095) / 4096;  // one block per 4096 keys at least
  unsigned hgrid = unsigned(ds->num_sms) * (hk->threads >= 1024 ? 1 : 2);
  if (work < hgrid) hgrid = unsigned(work > 0 ? work : 1);
  RS_CUDA(traced(T_HIST, n, s, [&] { return hk->launch(ha, hgrid, s); }), "launch upfront_hist");

  ScanArgs sa{hist, bases, force_all ? nullptr : ctrl + 4, n};
  RS_CUDA(traced(T_SCAN, 0, s, [&] { return scan_kernel(p.R)->launch(sa, unsigned(p.nd), s); }),
          "launch digit_scan");

  for (int j = 0; j < p.nd; ++j) {
    PassArgs pa{};
    pa.keys_in = keys_in;
    pa.keys_out = keys_out;
    pa.keys_alt = L.alt_k ? reinterpret_cast<uint32_t*>(temp + L.alt_k) : keys_out;
    pa.vals_in = vals_in;
    pa.vals_out = vals_out;
    pa.vals_alt = L.alt_v ? reinterpret_cast<uint32_t*>(temp + L.alt_v) : vals_out;
    pa.vals2_in = vals2_in;
    pa.vals2_out = vals2_out;
    pa.vals2_alt = vals2_alt;
    pa.n = n;
    pa.shift = p.dig[j].shift;
    pa.width = p.dig[j].width;
    pa.pass = j;
    pa.num_passes = p.nd;
    pa.bases = bases + size_t(j) * digits;
    pa.skip = force_all ? nullptr : ctrl + 4;
    pa.status = temp + L.status;
    pa.tile_counter = ctrl + j;
    pa.err = ds->err;
    pa.xin = p.xf;   // the first executed pass maps the input keys
    pa.xout = p.xf;  // the last one maps them back
    pa.pair_in = pair_vals_in;  // 64-bit values read and written interleaved
    pa.pair_out = pair_vals_out;
    // pass 0, when it runs, is the first executed pass: keys-only sorts rank it
    // without keeping the order of equal digits (there is none to keep yet)
    auto launch = (j == 0 && p.k->launch_first && !vals_in) ? p.k->launch_first : p.k->launch;
    RS_CUDA(traced(p.R == 8 ? T_PASS8 : T_PASS11, n, s, [&] { return launch(pa, pass_grid(p, ds), s); }),
            "launch onesweep");
  }
  return RS_OK;
}


// ---- the segmented pipeline (device-planned) ---------------------------------
// 8-bit digits over the low `nd` bytes of the keys; large segments go
// through tiled passes src -> (alt | dst) ... -> dst, tiny and small ones
// are sorted src -> dst in shared memory.
struct SegLayout {
  size_t counts = 0, seg_hist = 0, seg_bases = 0, large_seg = 0, tile_prefix = 0, small_seg = 0, tiny_seg = 0;
  size_t status = 0, jobs = 0, alt_k = 0, alt_v = 0, end = 0;
  size_t memset_from = 0, memset_bytes = 0;  // counts + seg_hist
  size_t tiles_ub = 0;
  int shape = 1;  // tiled-pass shape
};

// Shape of the segmented pipeline's tiled passes when a plan names none.
constexpr int kSegDefaultShape = 2;  // 384 x 20 tiles, three blocks per SM

SegLayout make_seg_layout(size_t off, uint32_t num_segs, uint64_t total_n, int nd, bool pairs,
                          int shape = kSegDefaultShape) {
  const SegKernels* sk = seg_kernels();
  SegLayout L;
  L.shape = shape;
  L.tiles_ub = size_t((total_n + sk->tile(pairs, shape) - 1) / sk->tile(pairs, shape)) + num_segs;
  off = align_up(off);
  L.counts = off;
  L.memset_from = off;
  off += align_up(size_t(kSegCountWords) * 4);
  L.seg_hist = off;
  off = align_up(off + size_t(num_segs) * nd * 256 * 4);
  L.memset_bytes = off - L.memset_from;
  L.seg_bases = off;
  off = align_up(off + size_t(num_segs) * nd * 256 * 4);
  L.large_seg = off;
  off = align_up(off + size_t(num_segs) * 4);
  L.tile_prefix = off;
  off = align_up(off + (size_t(num_segs) + 1) * 4);
  L.small_seg = off;
  off = align_up(off + size_t(num_segs) * 4);
  L.tiny_seg = off;
  off = align_up(off + size_t(num_segs) * 4);
  L.status = off;
  off = align_up(off + L.tiles_ub * 256 * 4);
  L.jobs = off;
  off = align_up(off + L.tiles_ub * sizeof(SegTileJob));
  L.alt_k = off;
  off = align_up(off + size_t(total_n) * 4);
  if (pairs) {
    L.alt_v = off;
    off = align_up(off + size_t(total_n) * 4);
  }
  L.end = off;
  return L;
}

// small_max: segments up to this many keys are sorted by one block in shared
// memory (at most the local sort's capacity); larger ones by tiled passes.
rs_status run_segmented(const SegLayout& L, unsigned char* temp, const uint32_t* kin, const uint32_t* vin,
                        uint32_t* kout, uint32_t* vout, const uint64_t* seg_off, uint32_t num_segs, int nd,
                        KeyXform xin, KeyXform xout, DeviceState* ds, cudaStream_t s, uint32_t small_max = 0) {
  const SegKernels* sk = seg_kernels();
  if (small_max == 0 || small_max > sk->small_max) small_max = sk->small_max;
  const uint32_t tiny_max = small_max < sk->tiny_max ? small_max : sk->tiny_max;
  const uint32_t seg_tile = sk->tile(vin != nullptr, L.shape);
  const bool pairs = vin != nullptr;
  uint32_t* counts = reinterpret_cast<uint32_t*>(temp + L.counts);
  const unsigned sms = unsigned(ds->num_sms);
  auto cap = [](size_t want, size_t limit) { return unsigned(want < limit ? (want > 0 ? want : 1) : limit); };
  RS_CUDA(traced(T_CLEAR, 0, s, [&] { return cudaMemsetAsync(temp + L.memset_from, 0, L.memset_bytes, s); }),
          "cudaMemsetAsync(segment counts)");
  SegPlanArgs pa{seg_off,
                 num_segs,
                 tiny_max,
                 small_max,
                 seg_tile,
                 reinterpret_cast<uint32_t*>(temp + L.large_seg),
                 reinterpret_cast<uint32_t*>(temp + L.tile_prefix),
                 reinterpret_cast<uint32_t*>(temp + L.small_seg),
                 reinterpret_cast<uint32_t*>(temp + L.tiny_seg),
                 counts};
  RS_CUDA(traced(T_SEGPLAN, 0, s, [&] { return launch_seg_plan(pa, s); }), "launch seg_plan");
  DigitSpec dig[kMaxDigits] = {};
  for (int j = 0; j < nd; ++j) dig[j] = DigitSpec{uint32_t(8 * j), 8u};
  SegHistArgs ha{};
  ha.keys = kin;
  ha.seg_off = seg_off;
  ha.large_seg = pa.large_seg;
  ha.tile_prefix = pa.tile_prefix;
  ha.counts = counts;
  ha.tile = seg_tile;
  ha.num_digits = nd;
  for (int j = 0; j < nd; ++j) ha.dig[j] = dig[j];
  ha.seg_hist = reinterpret_cast<uint32_t*>(temp + L.seg_hist);
  ha.status = reinterpret_cast<uint32_t*>(temp + L.status);
  ha.jobs = reinterpret_cast<SegTileJob*>(temp + L.jobs);
  ha.xform = xin;
  RS_CUDA(traced(T_SEGHIST, 0, s, [&] { return launch_seg_hist(ha, cap(L.tiles_ub, size_t(sms)), s); }),
          "launch seg_hist");
  SegScanArgs sa{ha.seg_hist, reinterpret_cast<uint32_t*>(temp + L.seg_bases), counts, nd};
  RS_CUDA(traced(T_SEGSCAN, 0, s, [&] { return launch_seg_scan(sa, cap(num_segs, size_t(sms) * 4), s); }),
          "launch seg_scan");
  uint32_t* alt_k = reinterpret_cast<uint32_t*>(temp + L.alt_k);
  uint32_t* alt_v = pairs ? reinterpret_cast<uint32_t*>(temp + L.alt_v) : nullptr;
  const uint32_t* src_k = kin;
  const uint32_t* src_v = vin;
  for (int p = 0; p < nd; ++p) {
    const bool to_out = ((nd - 1 - p) % 2) == 0;
    SegPassArgs ga{};
    ga.kin = src_k;
    ga.kout = to_out ? kout : alt_k;
    ga.vin = src_v;
    ga.vout = pairs ? (to_out ? vout : alt_v) : nullptr;
    ga.counts = counts;
    ga.seg_bases = sa.seg_bases;
    ga.jobs = ha.jobs;
    ga.num_digits = nd;
    ga.pass = p;
    ga.shift = dig[p].shift;
    ga.width = dig[p].width;
    ga.status = ha.status;
    ga.tile_counter = counts + SEG_TICKETS + p;
    ga.parity = uint32_t(p & 1) ^ 1u;
    ga.err = ds->err;
    ga.xin = p == 0 ? xin : kIdentityXform;
    ga.xout = p == nd - 1 ? xout : kIdentityXform;
    RS_CUDA(traced(T_SEGPASS, 0, s,
                   [&] {
                     return launch_seg_pass(ga, pairs, L.shape,
                                            cap(L.tiles_ub, size_t(sms) * sk->blocks_per_sm[L.shape]), s);
                   }),
            "launch seg_pass");
    src_k = ga.kout;
    src_v = ga.vout;
  }
  LocalArgs la{};
  la.kin = kin;
  la.kout = kout;
  la.vin = vin;
  la.vout = vout;
  la.seg_off = seg_off;
  la.num_digits = nd;
  for (int j = 0; j < nd; ++j) la.dig[j] = dig[j];
  la.xin = xin;
  la.xout = xout;
  la.list = pa.tiny_seg;
  la.count = counts + SEG_NUM_TINY;
  RS_CUDA(traced(T_LOCAL, 0, s, [&] { return launch_local_sort(la, false, pairs, cap(num_segs, size_t(sms) * 8), s); }),
          "launch local_sort (tiny)");
  la.list = pa.small_seg;
  la.count = counts + SEG_NUM_SMALL;
  RS_CUDA(traced(T_LOCAL, 0, s, [&] { return launch_local_sort(la, true, pairs, cap(num_segs, size_t(sms) * 2), s); }),
          "launch local_sort (small)");
  return RS_OK;
}

rs_status check_common(const void* keys_in, const void* keys_out, uint64_t n, void* temp, size_t* temp_bytes) {
  if (!temp_bytes) return fail(RS_ERR_INVALID, "temp_bytes is NULL");
  if (n >= (uint64_t(1) << 32)) return fail(RS_ERR_INVALID, "n = %llu: must be below 2^32", (unsigned long long)n);
  if (temp && (reinterpret_cast<uintptr_t>(temp) % kAlign)) return fail(RS_ERR_INVALID, "temp is not 256-byte aligned");
  if (n > 0 && temp) {
    if (!keys_in || !keys_out) return fail(RS_ERR_INVALID, "NULL key buffer");
    if ((reinterpret_cast<uintptr_t>(keys_in) | reinterpret_cast<uintptr_t>(keys_out)) & 3)
      return fail(RS_ERR_INVALID, "key buffers must be 4-byte aligned");
  }
  return RS_OK;
}


// ---- the MSD plan ---------------------------------------------------------------
// Bucketing by the keys' bits 18-31 (2^14 buckets), then the segmented
// pipeline on the buckets over the three low bytes: a one-block local sort
// for buckets of up to 16,384 keys, tiled passes for larger ones.
//   keys only:  count per (chunk, bucket) [msd.cu] -> column and base scans
//               -> one distribution pass [msd.cu] -> segmented pipeline;
//   key+value:  two stable LSD passes over bits 18-24 and 25-31 (the
//               distribution must keep equal keys in input order), the same
//               count and scans for the bucket offsets -> segmented pipeline.
constexpr uint32_t kMsdChunks = 304;  // blocks of the count and distribution kernels
constexpr uint32_t kMsdBuckets = 1u << (32 - kMsdShift);

struct MsdLayout {
  Layout lsd;             // key+value: control, histograms, status and alternate buffers of the two passes
  SortPlan q;             // key+value: the two-pass plan
  size_t bk = 0, bv = 0;  // bucket buffers (keys, values)
  size_t mhist = 0, mtot = 0, seg_off = 0;
  SegLayout seg;
  size_t total = 0;
};

rs_status make_msd_layout(const SortPlan& p, uint64_t n, bool pairs, MsdLayout* out) {
  MsdLayout M;
  size_t off = 0;
  if (pairs) {
    M.q = p;
    M.q.msd = false;
    M.q.nd = 2;
    M.q.dig[0] = DigitSpec{kMsdShift, 7u};
    M.q.dig[1] = DigitSpec{kMsdShift + 7u, 32u - kMsdShift - 7u};
    if (rs_status st = pick_kernel(8, 1, 1, needs_wide_status(n), &M.q.k); st != RS_OK) return st;
    M.q.num_tiles = (n + M.q.k->tile - 1) / M.q.k->tile;
    M.lsd = make_layout(M.q, n, true);
    off = M.lsd.total;
  }
  M.bk = off;
  off = align_up(off + size_t(n) * 4);
  if (pairs) {
    M.bv = off;
    off = align_up(off + size_t(n) * 4);
  }
  M.mhist = off;
  off = align_up(off + size_t(kMsdChunks) * kMsdBuckets * 4);
  M.mtot = off;
  off = align_up(off + size_t(kMsdBuckets) * 4);
  M.seg_off = off;
  off = align_up(off + (size_t(kMsdBuckets) + 1) * 8);
  M.seg = make_seg_layout(off, kMsdBuckets, n, 3, pairs);
  M.total = M.seg.end;
  *out = M;
  return RS_OK;
}

rs_status run_msd(const SortPlan& p, const MsdLayout& M, const uint32_t* keys_in, const uint32_t* vals_in,
                  uint32_t* keys_out, uint32_t* vals_out, uint32_t n, unsigned char* temp, DeviceState* ds,
                  cudaStream_t s) {
  const bool pairs = vals_in != nullptr;
  uint32_t* bk = reinterpret_cast<uint32_t*>(temp + M.bk);
  uint32_t* bv = pairs ? reinterpret_cast<uint32_t*>(temp + M.bv) : nullptr;
  MsdArgs ma{};
  ma.keys = keys_in;
  ma.n = n;
  ma.x = p.xf;
  ma.chunks = kMsdChunks;
  ma.hist = reinterpret_cast<uint32_t*>(temp + M.mhist);
  ma.totals = reinterpret_cast<uint32_t*>(temp + M.mtot);
  ma.seg_off = reinterpret_cast<uint64_t*>(temp + M.seg_off);
  ma.out = bk;
  ma.err = ds->err;
  RS_CUDA(traced(T_MSDCOUNT, n, s, [&] { return launch_msd_count(ma, s); }), "launch msd_count");
  RS_CUDA(traced(T_MSDSCAN, 0, s, [&] { return launch_msd_scan(ma, s); }), "launch msd_scan");
  if (!pairs) {
    RS_CUDA(traced(T_MSDSCATTER, n, s, [&] { return launch_msd_scatter(ma, s); }), "launch msd_scatter");
    // the bucket buffer holds order-mapped keys; the local phase maps them back
    return run_segmented(M.seg, temp, bk, nullptr, keys_out, nullptr, ma.seg_off, kMsdBuckets, 3, kIdentityXform,
                         p.xf, ds, s);
  }
  if (rs_status st = run_lsd(M.q, M.lsd, keys_in, vals_in, bk, bv, n, temp, true, ds, s); st != RS_OK) return st;
  return run_segmented(M.seg, temp, bk, bv, keys_out, vals_out, ma.seg_off, kMsdBuckets, 3, p.xf, p.xf, ds, s);
}

// ---- the single-launch sort -----------------------------------------------------
// Up to (resident blocks) x 9,216 keys with the automatic plan: clear + one
// cooperative launch instead of clear + histogram + scans + four passes.  It
// uses the LSD layout's control words (word 12: the barrier counter), digit
// histograms, status rows (the layout holds a row per tile of the smallest
// shape up to kFusedStatusMaxKeys keys) and alternate buffers.
constexpr uint64_t kFusedStatusMaxKeys = uint64_t(1) << 22;
rs_status run_fused(const SortPlan& p, const Layout& L, const uint32_t* keys_in, const uint32_t* vals_in,
                    uint32_t* keys_out, uint32_t* vals_out, uint32_t n, int shape, unsigned char* temp,
                    DeviceState* ds, cudaStream_t s) {
  const bool pairs = vals_in != nullptr;
  const uint32_t tiles = (n + fused_tile_keys(shape) - 1) / fused_tile_keys(shape);
  if (size_t(tiles) * 256 * 4 > L.status_bytes) return fail(RS_ERR_CUDA, "single-launch sort: status too small");
  RS_CUDA(traced(T_CLEAR, 0, s, [&] { return cudaMemsetAsync(temp, 0, L.status + size_t(tiles) * 256 * 4, s); }),
          "cudaMemsetAsync(temp)");
  FusedArgs a{};
  a.keys_in = keys_in;
  a.keys_out = keys_out;
  a.keys_alt = L.alt_k ? reinterpret_cast<uint32_t*>(temp + L.alt_k) : keys_out;
  a.vals_in = vals_in;
  a.vals_out = vals_out;
  a.vals_alt = pairs && L.alt_v ? reinterpret_cast<uint32_t*>(temp + L.alt_v) : vals_out;
  a.n = n;
  a.xf = p.xf;
  a.hist = reinterpret_cast<uint32_t*>(temp + L.hist);
  a.status = temp + L.status;
  a.bar = reinterpret_cast<uint32_t*>(temp + L.ctrl) + 12;
  a.err = ds->err;
  RS_CUDA(traced(T_FUSED, n, s, [&] { return launch_fused(a, tiles, pairs, shape, s); }), "launch fused sort");
  return RS_OK;
}

rs_status sort_impl(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out, uint32_t* vals_out,
                    uint64_t n, uint32_t num_parts, uint64_t* h_part_offsets, const rs_plan* user_plan, void* temp,
                    size_t* temp_bytes, cudaStream_t s, bool pairs) {
  g_last_error.clear();
  const rs_plan eff = resolve_plan(pairs ? RS_ENTRY_SORT_U32_PAIRS : RS_ENTRY_SORT_U32, n, user_plan);
  const rs_plan* plan = &eff;
  rs_status st = check_common(keys_in, keys_out, n, temp, temp_bytes);
  if (st != RS_OK) return st;
  if (num_parts < 1) return fail(RS_ERR_INVALID, "num_parts must be >= 1");
  SortPlan p;
  st = make_plan(n, pairs, plan, &p);
  if (st != RS_OK) return st;
  const bool automatic = plan->digit_bits == 0 && plan->mode == RS_MODE_AUTO && plan->tile == 0;
  const bool fusable = automatic && p.R == 8 && p.nd == 4 && !p.msd && !p.k->wide_status;
  if (fusable && n <= kFusedStatusMaxKeys)  // status rows for the single-launch sort's smallest tiles
    p.status_rows = size_t((n + fused_tile_keys(kFusedShapes - 1) - 1) / fused_tile_keys(kFusedShapes - 1));
  Layout L = make_layout(p, n, pairs);
  MsdLayout M;
  if (p.msd) {
    if (rs_status st2 = make_msd_layout(p, n, pairs, &M); st2 != RS_OK) return st2;
    L.total = M.total;
  }
  if (!temp) {
    *temp_bytes = L.total;
    return RS_OK;
  }
  if (*temp_bytes < L.total)
    return fail(RS_ERR_TEMP_TOO_SMALL, "temp_bytes = %zu, need %zu", *temp_bytes, L.total);
  if (pairs && n > 0) {
    if (!vals_in || !vals_out) return fail(RS_ERR_INVALID, "NULL value buffer");
    if ((reinterpret_cast<uintptr_t>(vals_in) | reinterpret_cast<uintptr_t>(vals_out)) & 3)
      return fail(RS_ERR_INVALID, "value buffers must be 4-byte aligned");
  }
  const size_t nb = size_t(n) * 4;
  const void* outs[2] = {keys_out, pairs ? vals_out : nullptr};
  const void* all[4] = {keys_in, pairs ? vals_in : nullptr, keys_out, pairs ? vals_out : nullptr};
  for (const void* o : outs) {
    if (!o) continue;
    for (const void* x : all)
      if (x && x != o && overlaps(o, nb, x, nb)) return fail(RS_ERR_INVALID, "an output overlaps another buffer");
    if (o == keys_in || (pairs && o == vals_in)) return fail(RS_ERR_INVALID, "an output aliases an input");
    if (overlaps(o, nb, temp, L.total)) return fail(RS_ERR_INVALID, "an output overlaps temp");
  }
  if (pairs && n > 0 && keys_out == vals_out) return fail(RS_ERR_INVALID, "keys_out and vals_out alias");
  for (const void* x : all)
    if (overlaps(x, nb, temp, L.total)) return fail(RS_ERR_INVALID, "a buffer overlaps temp");
  if (h_part_offsets) part_offsets_host(n, num_parts, h_part_offsets);
  if (n == 0) return RS_OK;
  DeviceState* ds = nullptr;
  st = device_state(&ds);
  if (st != RS_OK) return st;
  if (p.msd)
    return run_msd(p, M, keys_in, pairs ? vals_in : nullptr, keys_out, pairs ? vals_out : nullptr, uint32_t(n),
                   static_cast<unsigned char*>(temp), ds, s);
  // A small array with the automatic plan fits one block: every digit is
  // sorted in shared memory by one launch (no histogram, scans or tiled
  // passes), which is several times faster for such sizes.
  const SegKernels* sk = seg_kernels();
  if (automatic && n <= sk->small_max) {
    LocalArgs la{};
    la.kin = keys_in;
    la.kout = keys_out;
    la.vin = pairs ? vals_in : nullptr;
    la.vout = pairs ? vals_out : nullptr;
    la.single_n = uint32_t(n);
    la.num_digits = 4;
    for (int j = 0; j < 4; ++j) la.dig[j] = DigitSpec{uint32_t(8 * j), 8u};
    la.xin = p.xf;
    la.xout = p.xf;
    RS_CUDA(traced(T_LOCAL, double(n), s, [&] { return launch_local_sort(la, n > sk->tiny_max, pairs, 1u, s); }),
            "launch local_sort (one array)");
    return RS_OK;
  }
  // Up to a few million keys: every tile resident at once, the whole sort in
  // one launch (8-bit digits, the same passes).  The tile shape: the smallest
  // whose tiles still number at most one per SM, else the largest.
  if (fusable) {
    int sh = 0;
    for (int c = kFusedShapes - 1; c > 0; --c)
      if ((n + fused_tile_keys(c) - 1) / fused_tile_keys(c) <= uint64_t(ds->num_sms)) {
        sh = c;
        break;
      }
    const size_t tiles = (n + fused_tile_keys(sh) - 1) / fused_tile_keys(sh);
    if (tiles <= ds->fused_tiles[pairs ? 1 : 0][sh] && tiles * 1024 <= L.status_bytes)
      return run_fused(p, L, keys_in, pairs ? vals_in : nullptr, keys_out, pairs ? vals_out : nullptr, uint32_t(n),
                       sh, static_cast<unsigned char*>(temp), ds, s);
  }
  return run_lsd(p, L, keys_in, pairs ? vals_in : nullptr, keys_out, pairs ? vals_out : nullptr, uint32_t(n),
                 static_cast<unsigned char*>(temp), false, ds, s);
}

// ---- 64-bit keys -----------------------------------------------------------------
// Eight 8-bit digits; the key+payload pass kernel moves both words of every
// key (low word as the key for digits 0-3, high word for digits 4-7).  With a
// tiled (non-persistent) pass kernel the histograms and the first executed
// pass read the interleaved keys and the last one writes them (fused); the
// persistent kernels take word planes made by a split kernel and joined back
// at the end.
struct Layout64 {
  bool fused = false;
  size_t ctrl = 0;    // [0, 8): tile tickets of the 8 passes; [8, 16): skip flags
  size_t hist = 0;    // [8][256]
  size_t bases = 0;   // [8][256]
  size_t status = 0, status_bytes = 0;
  size_t plane[6] = {};  // lo/hi words of the output, alternate and (split only) input order
  size_t val_alt = 0;    // the values' alternate plane (key+value sorts)
  size_t idx_out = 0;    // 64-bit values: the index plane of the output order
  size_t memset_bytes = 0, total = 0;
};

Layout64 make_layout64(const SortPlan& p, uint64_t n, bool pairs, bool vals64 = false) {
  Layout64 L;
  L.fused = pair_io_kernel(p.k) != nullptr;
  size_t off = 0;
  L.ctrl = off;
  off += kAlign;
  L.hist = off;
  off = align_up(off + 8 * 256 * 4);
  L.memset_bytes = off;
  L.bases = off;
  off = align_up(off + 8 * 256 * 4);
  L.status = off;
  L.status_bytes = p.num_tiles * 256 * (p.k->wide_status ? 8 : 4);
  off = align_up(off + L.status_bytes);
  for (int i = 0; i < (L.fused ? 4 : 6); ++i) {
    L.plane[i] = off;
    off = align_up(off + size_t(n) * 4);
  }
  if (pairs) {
    L.val_alt = off;
    off = align_up(off + size_t(n) * 4);
  }
  if (vals64) {
    L.idx_out = off;
    off = align_up(off + size_t(n) * 4);
  }
  L.total = off;
  return L;
}

rs_status key_xform64(const rs_plan* user, KeyXform64* out) {
  const uint32_t kind = user ? user->key_kind : uint32_t(RS_KEY_U32);
  switch (kind) {
    case RS_KEY_U32: *out = KeyXform64{0u, 0u, 0u}; return RS_OK;
    case RS_KEY_I32: *out = KeyXform64{0u, 0u, 0x80000000u}; return RS_OK;
    case RS_KEY_F32: *out = KeyXform64{0xffffffffu, 0x7fffffffu, 0x80000000u}; return RS_OK;
    default: return fail(RS_ERR_INVALID, "unknown key_kind %u", kind);
  }
}

// vals64_in/out (fused layouts only): 64-bit values, sorted through an input
// index that the passes carry as their second payload word.
rs_status run_lsd64(const SortPlan& p, const Layout64& L, const uint64_t* keys_in, const uint32_t* vals_in,
                    uint64_t* keys_out, uint32_t* vals_out, uint32_t n, KeyXform64 x, unsigned char* temp,
                    DeviceState* ds, cudaStream_t s, const uint64_t* vals64_in = nullptr,
                    uint64_t* vals64_out = nullptr) {
  uint32_t* ctrl = reinterpret_cast<uint32_t*>(temp + L.ctrl);
  uint32_t* hist = reinterpret_cast<uint32_t*>(temp + L.hist);
  uint32_t* bases = reinterpret_cast<uint32_t*>(temp + L.bases);
  uint32_t* pl[6] = {};
  for (int i = 0; i < (L.fused ? 4 : 6); ++i) pl[i] = reinterpret_cast<uint32_t*>(temp + L.plane[i]);
  const OnesweepKernel* pk = L.fused ? pair_io_kernel(p.k) : p.k;
  uint32_t *lo_out = pl[0], *hi_out = pl[1], *lo_alt = pl[2], *hi_alt = pl[3], *lo_in = pl[4], *hi_in = pl[5];
  const uint2* k2 = reinterpret_cast<const uint2*>(keys_in);
  RS_CUDA(traced(T_CLEAR, 0, s, [&] { return cudaMemsetAsync(temp, 0, L.memset_bytes, s); }),
          "cudaMemsetAsync(temp)");
  const unsigned egrid = unsigned(std::min<size_t>((size_t(n) + 255) / 256, size_t(ds->num_sms) * 8));
  if (!L.fused) {
    WideArgs wa{k2, reinterpret_cast<uint2*>(keys_out), lo_in, hi_in, n, x};
    RS_CUDA(traced(T_SPLIT, n, s, [&] { return launch_split64(wa, egrid, s); }), "launch split64");
  }
  // the eight digit histograms: four per word
  const HistKernel* hk = hist_kernel(8);
  const size_t work = (size_t(n) + 4095) / 4096;
  unsigned hgrid = unsigned(ds->num_sms);
  if (work < hgrid) hgrid = unsigned(work > 0 ? work : 1);
  if (L.fused) {  // one read of the interleaved keys
    HistArgs ha{};
    ha.keys64 = k2;
    ha.x64 = x;
    ha.n = n;
    ha.hist = hist;
    ha.zero_ptr = reinterpret_cast<uint4*>(temp + L.status);
    ha.zero_vec4 = L.status_bytes / 16;
    RS_CUDA(traced(T_HIST, n, s, [&] { return launch_hist64(ha, hgrid, s); }), "launch upfront_hist64");
  }
  for (int w = 0; w < (L.fused ? 0 : 2); ++w) {
    HistArgs ha{};
    ha.keys = w == 0 ? lo_in : hi_in;
    ha.n = n;
    ha.num_digits = 4;
    for (int j = 0; j < 4; ++j) ha.dig[j] = DigitSpec{uint32_t(8 * j), 8u};
    ha.hist = hist + size_t(w) * 4 * 256;
    ha.zero_ptr = w == 0 ? reinterpret_cast<uint4*>(temp + L.status) : nullptr;
    ha.zero_vec4 = w == 0 ? L.status_bytes / 16 : 0;
    RS_CUDA(traced(T_HIST, n, s, [&] { return hk->launch(ha, hgrid, s); }), "launch upfront_hist");
  }
  ScanArgs sa{hist, bases, ctrl + 8, n};
  RS_CUDA(traced(T_SCAN, 0, s, [&] { return scan_kernel(8)->launch(sa, 8u, s); }), "launch digit_scan");
  for (int j = 0; j < 8; ++j) {
    const bool high = j >= 4;  // which word carries the digit
    PassArgs pa{};
    pa.keys_in = high ? hi_in : lo_in;
    pa.keys_out = high ? hi_out : lo_out;
    pa.keys_alt = high ? hi_alt : lo_alt;
    pa.vals_in = high ? lo_in : hi_in;
    pa.vals_out = high ? lo_out : hi_out;
    pa.vals_alt = high ? lo_alt : hi_alt;
    if (vals_in) {  // the values ride as a second payload word, from and into the caller's arrays
      pa.vals2_in = vals_in;
      pa.vals2_out = vals_out;
      pa.vals2_alt = reinterpret_cast<uint32_t*>(temp + L.val_alt);
    } else if (vals64_in) {  // so does the input index of a 64-bit value
      pa.vals2_out = reinterpret_cast<uint32_t*>(temp + L.idx_out);
      pa.vals2_alt = reinterpret_cast<uint32_t*>(temp + L.val_alt);
      pa.iota = 1;
      pa.gather = reinterpret_cast<const uint2*>(vals64_in);
      pa.gather_out = reinterpret_cast<uint2*>(vals64_out);
    }
    pa.n = n;
    pa.shift = uint32_t(8 * (j % 4));
    pa.width = 8;
    pa.pass = j;
    pa.num_passes = 8;
    pa.bases = bases + size_t(j) * 256;
    pa.skip = ctrl + 8;
    pa.status = temp + L.status;
    pa.tile_counter = ctrl + j;
    pa.err = ds->err;
    pa.xin = kIdentityXform;   // the planes hold mapped words
    pa.xout = kIdentityXform;
    if (L.fused) {  // the first executed pass reads the keys, the last one writes them
      pa.pair_in = k2;
      pa.pair_out = reinterpret_cast<uint2*>(keys_out);
      pa.pair_key = 1;
      pa.key_high = high ? 1u : 0u;
      pa.x64 = x;
    }
    RS_CUDA(traced(T_PASS8, n, s, [&] { return pk->launch(pa, pass_grid(p, ds), s); }), "launch onesweep (64-bit)");
  }
  if (!L.fused) {  // the last executed pass always writes the output planes
    WideArgs ja{nullptr, reinterpret_cast<uint2*>(keys_out), lo_out, hi_out, n, x};
    RS_CUDA(traced(T_JOIN, n, s, [&] { return launch_join64(ja, egrid, s); }), "launch join64");
  }
  return RS_OK;
}

// Partition offsets of every segment, absolute (segment start added).
__global__ void seg_part_offsets_kernel(const uint64_t* seg, uint32_t num_segs, uint32_t parts, uint64_t* out) {
  const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const size_t per = size_t(parts) + 1;
  if (i >= size_t(num_segs) * per) return;
  const size_t sidx = i / per;
  const uint64_t p = i % per;
  const uint64_t a = seg[sidx], m = seg[sidx + 1] - a;
  const uint64_t q = m / parts, r = m % parts;
  out[i] = a + p * q + (p < r ? p : r);
}

}  // namespace

void set_last_error(int /*status*/, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

}  // namespace rs

using namespace rs;

extern "C" {

rs_status rs_sort_u32(const uint32_t* keys_in, uint32_t* keys_out, uint64_t n, uint32_t num_parts,
                      uint64_t* h_part_offsets, const rs_plan* plan, void* temp, size_t* temp_bytes,
                      rs_stream_t stream) {
  return sort_impl(keys_in, nullptr, keys_out, nullptr, n, num_parts, h_part_offsets, plan, temp, temp_bytes,
                   reinterpret_cast<cudaStream_t>(stream), false);
}

rs_status rs_sort_u32_pairs(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out,
                            uint32_t* vals_out, uint64_t n, uint32_t num_parts, uint64_t* h_part_offsets,
                            const rs_plan* plan, void* temp, size_t* temp_bytes, rs_stream_t stream) {
  return sort_impl(keys_in, vals_in, keys_out, vals_out, n, num_parts, h_part_offsets, plan, temp, temp_bytes,
                   reinterpret_cast<cudaStream_t>(stream), true);
}

// vbytes: 0 (keys only), 4 (uint32 values) or 8 (uint64 values).
static rs_status sort64_impl(const uint64_t* keys_in, const void* vals_in, uint64_t* keys_out, void* vals_out,
                             uint64_t n, uint32_t num_parts, uint64_t* h_part_offsets, const rs_plan* plan,
                             void* temp, size_t* temp_bytes, rs_stream_t stream, int vbytes) {
  const bool pairs = vbytes != 0;
  g_last_error.clear();
  const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (!temp_bytes) return fail(RS_ERR_INVALID, "temp_bytes is NULL");
  if (n >= (uint64_t(1) << 32)) return fail(RS_ERR_INVALID, "n = %llu: must be below 2^32", (unsigned long long)n);
  if (num_parts < 1) return fail(RS_ERR_INVALID, "num_parts must be >= 1");
  if (plan && plan->digit_bits && plan->digit_bits != 8)
    return fail(RS_ERR_UNSUPPORTED, "64-bit keys use 8-bit digits");
  if (plan && plan->mode == RS_MODE_MSD) return fail(RS_ERR_UNSUPPORTED, "64-bit keys use the LSD plan");
  KeyXform64 x;
  if (rs_status st = key_xform64(plan, &x); st != RS_OK) return st;
  rs_plan q = plan ? *plan : rs_plan{0, 0, 0, 0};
  q.digit_bits = 8;
  q.mode = RS_MODE_LSD;
  q.key_kind = RS_KEY_U32;
  // the shapes with interleaved-word pass kernels: 384 x 24 (three blocks per
  // SM) for keys alone above 2^22 keys (GB300, 2^26 keys: 335 us per pass
  // against 349 at 512 x 24; 2^23: 20.0 against 18.7 Gkeys/s), else 512 x 16
  // (the one with 64-bit status words and two payload words)
  if (q.tile == 0) q.tile = (vbytes == 0 && n > (uint64_t(1) << 22) && !needs_wide_status(n)) ? 8u : 1u;
  SortPlan p;
  if (rs_status st = make_plan(n, true, &q, &p, pairs ? 2 : 1); st != RS_OK) return st;
  const Layout64 L = make_layout64(p, n, pairs, vbytes == 8);
  if (vbytes == 8 && !L.fused)
    return fail(RS_ERR_UNSUPPORTED, "64-bit values: tile shape %u has no interleaved pass kernel", q.tile);
  if (!temp) {
    *temp_bytes = L.total;
    return RS_OK;
  }
  if (reinterpret_cast<uintptr_t>(temp) % kAlign) return fail(RS_ERR_INVALID, "temp is not 256-byte aligned");
  if (*temp_bytes < L.total) return fail(RS_ERR_TEMP_TOO_SMALL, "temp_bytes = %zu, need %zu", *temp_bytes, L.total);
  const size_t nb = size_t(n) * 8;
  if (n > 0) {
    if (!keys_in || !keys_out) return fail(RS_ERR_INVALID, "NULL key buffer");
    if ((reinterpret_cast<uintptr_t>(keys_in) | reinterpret_cast<uintptr_t>(keys_out)) & 7)
      return fail(RS_ERR_INVALID, "64-bit key buffers must be 8-byte aligned");
    if (overlaps(keys_out, nb, keys_in, nb)) return fail(RS_ERR_INVALID, "keys_out overlaps keys_in");
    if (overlaps(keys_out, nb, temp, L.total) || overlaps(keys_in, nb, temp, L.total))
      return fail(RS_ERR_INVALID, "a key buffer overlaps temp");
    if (pairs) {
      const size_t vb = size_t(n) * vbytes;
      if (!vals_in || !vals_out) return fail(RS_ERR_INVALID, "NULL value buffer");
      if ((reinterpret_cast<uintptr_t>(vals_in) | reinterpret_cast<uintptr_t>(vals_out)) & (vbytes - 1))
        return fail(RS_ERR_INVALID, "value buffers must be %d-byte aligned", vbytes);
      if (overlaps(vals_out, vb, vals_in, vb) || overlaps(vals_out, vb, keys_in, nb) ||
          overlaps(vals_out, vb, keys_out, nb) || overlaps(vals_out, vb, temp, L.total) ||
          overlaps(keys_out, nb, vals_in, vb))
        return fail(RS_ERR_INVALID, "an output overlaps another buffer");
    }
  }
  if (h_part_offsets) part_offsets_host(n, num_parts, h_part_offsets);
  if (n == 0) return RS_OK;
  DeviceState* ds = nullptr;
  if (rs_status st = device_state(&ds); st != RS_OK) return st;
  if (vbytes == 8)
    return run_lsd64(p, L, keys_in, nullptr, keys_out, nullptr, uint32_t(n), x, static_cast<unsigned char*>(temp), ds,
                     s, static_cast<const uint64_t*>(vals_in), static_cast<uint64_t*>(vals_out));
  return run_lsd64(p, L, keys_in, static_cast<const uint32_t*>(vals_in), keys_out, static_cast<uint32_t*>(vals_out),
                   uint32_t(n), x, static_cast<unsigned char*>(temp), ds, s);
}

rs_status rs_sort_u64(const uint64_t* keys_in, uint64_t* keys_out, uint64_t n, uint32_t num_parts,
                      uint64_t* h_part_offsets, const rs_plan* plan, void* temp, size_t* temp_bytes,
                      rs_stream_t stream) {
  return sort64_impl(keys_in, nullptr, keys_out, nullptr, n, num_parts, h_part_offsets, plan, temp, temp_bytes,
                     stream, 0);
}

rs_status rs_sort_u64_pairs(const uint64_t* keys_in, const uint32_t* vals_in, uint64_t* keys_out,
                            uint32_t* vals_out, uint64_t n, uint32_t num_parts, uint64_t* h_part_offsets,
                            const rs_plan* plan, void* temp, size_t* temp_bytes, rs_stream_t stream) {
  return sort64_impl(keys_in, vals_in, keys_out, vals_out, n, num_parts, h_part_offsets, plan, temp, temp_bytes,
                     stream, 4);
}

rs_status rs_sort_u64_pairs64(const uint64_t* keys_in, const uint64_t* vals_in, uint64_t* keys_out,
                              uint64_t* vals_out, uint64_t n, uint32_t num_parts, uint64_t* h_part_offsets,
                              const rs_plan* plan, void* temp, size_t* temp_bytes, rs_stream_t stream) {
  return sort64_impl(keys_in, vals_in, keys_out, vals_out, n, num_parts, h_part_offsets, plan, temp, temp_bytes,
                     stream, 8);
}

rs_status rs_sort_u32_pairs64(const uint32_t* keys_in, const uint64_t* vals_in, uint32_t* keys_out,
                              uint64_t* vals_out, uint64_t n, uint32_t num_parts, uint64_t* h_part_offsets,
                              const rs_plan* plan, void* temp, size_t* temp_bytes, rs_stream_t stream) {
  g_last_error.clear();
  const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  rs_status st = check_common(keys_in, keys_out, n, temp, temp_bytes);
  if (st != RS_OK) return st;
  if (num_parts < 1) return fail(RS_ERR_INVALID, "num_parts must be >= 1");
  if (plan && plan->mode == RS_MODE_MSD) return fail(RS_ERR_UNSUPPORTED, "64-bit values use the LSD plan");
  if (plan && plan->digit_bits && plan->digit_bits != 8) return fail(RS_ERR_UNSUPPORTED, "64-bit values use 8-bit digits");
  rs_plan q = plan ? *plan : rs_plan{0, 0, 0, 0};
  q.digit_bits = 8;
  q.mode = RS_MODE_LSD;
  if (q.tile == 0) q.tile = 1;  // the shape with two-payload-word pass kernels
  SortPlan p;
  if ((st = make_plan(n, true, &q, &p, 2)) != RS_OK) return st;
  // the sort's own layout (keys, the low value words as the first payload
  // plane) followed by the value planes: low and high words of the output,
  // the high words' alternate plane and (split only) both words of the input.
  // A tiled pass kernel reads and writes the interleaved values itself
  // (fused); a persistent one takes planes split and joined by kernels.
  Layout L = make_layout(p, n, true);
  const bool fused = pair_io_kernel(p.k) != nullptr;
  const int nplanes = fused ? 3 : 5;
  size_t plane[5] = {};
  size_t off = L.total;
  for (int i = 0; i < nplanes; ++i) {
    plane[i] = off;
    off = align_up(off + size_t(n) * 4);
  }
  const size_t need = off;
  if (!temp) {
    *temp_bytes = need;
    return RS_OK;
  }
  if (*temp_bytes < need) return fail(RS_ERR_TEMP_TOO_SMALL, "temp_bytes = %zu, need %zu", *temp_bytes, need);
  const size_t kb = size_t(n) * 4, vb = size_t(n) * 8;
  if (n > 0) {
    if (!vals_in || !vals_out) return fail(RS_ERR_INVALID, "NULL value buffer");
    if ((reinterpret_cast<uintptr_t>(vals_in) | reinterpret_cast<uintptr_t>(vals_out)) & 7)
      return fail(RS_ERR_INVALID, "64-bit value buffers must be 8-byte aligned");
    if (overlaps(keys_out, kb, keys_in, kb) || overlaps(keys_out, kb, vals_in, vb) ||
        overlaps(vals_out, vb, keys_in, kb) || overlaps(vals_out, vb, vals_in, vb) ||
        overlaps(vals_out, vb, keys_out, kb) || overlaps(keys_out, kb, temp, need) ||
        overlaps(vals_out, vb, temp, need) || overlaps(keys_in, kb, temp, need) || overlaps(vals_in, vb, temp, need))
      return fail(RS_ERR_INVALID, "a buffer overlaps another");
  }
  if (h_part_offsets) part_offsets_host(n, num_parts, h_part_offsets);
  if (n == 0) return RS_OK;
  DeviceState* ds = nullptr;
  if ((st = device_state(&ds)) != RS_OK) return st;
  unsigned char* t = static_cast<unsigned char*>(temp);
  uint32_t* pl[5] = {};
  for (int i = 0; i < nplanes; ++i) pl[i] = reinterpret_cast<uint32_t*>(t + plane[i]);
  uint32_t *vlo_out = pl[0], *vhi_out = pl[1], *vhi_alt = pl[2], *vlo_in = pl[3], *vhi_in = pl[4];
  if (fused) {
    SortPlan q2 = p;
    q2.k = pair_io_kernel(p.k);
    return run_lsd(q2, L, keys_in, nullptr, keys_out, vlo_out, uint32_t(n), t, false, ds, s, nullptr, vhi_out,
                   vhi_alt, reinterpret_cast<const uint2*>(vals_in), reinterpret_cast<uint2*>(vals_out));
  }
  const unsigned egrid = unsigned(std::min<size_t>((size_t(n) + 255) / 256, size_t(ds->num_sms) * 8));
  const KeyXform64 ident{0u, 0u, 0u};
  WideArgs wa{reinterpret_cast<const uint2*>(vals_in), nullptr, vlo_in, vhi_in, n, ident};
  RS_CUDA(traced(T_SPLIT, double(n), s, [&] { return launch_split64(wa, egrid, s); }), "launch split64 (values)");
  st = run_lsd(p, L, keys_in, vlo_in, keys_out, vlo_out, uint32_t(n), t, false, ds, s, vhi_in, vhi_out, vhi_alt);
  if (st != RS_OK) return st;
  WideArgs ja{nullptr, reinterpret_cast<uint2*>(vals_out), vlo_out, vhi_out, n, ident};
  RS_CUDA(traced(T_JOIN, double(n), s, [&] { return launch_join64(ja, egrid, s); }), "launch join64 (values)");
  return RS_OK;
}

rs_status rs_merge_u32(const uint32_t* a, const uint32_t* va, uint64_t na, const uint32_t* b, const uint32_t* vb,
                       uint64_t nb, uint32_t* out, uint32_t* vout, uint32_t num_parts, uint64_t* h_part_offsets,
                       const rs_plan* plan, void* temp, size_t* temp_bytes, rs_stream_t stream) {
  g_last_error.clear();
  const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (!temp_bytes) return fail(RS_ERR_INVALID, "temp_bytes is NULL");
  const uint64_t n = na + nb;
  if (na >= (uint64_t(1) << 32) || nb >= (uint64_t(1) << 32) || n >= (uint64_t(1) << 32))
    return fail(RS_ERR_INVALID, "na + nb must be below 2^32");
  if (num_parts < 1) return fail(RS_ERR_INVALID, "num_parts must be >= 1");
  // payloads: all three arrays, or none (a run with no elements may pass NULL)
  const bool pairs = va || vb || vout;
  if (pairs && ((na && !va) || (nb && !vb) || (na + nb && !vout)))
    return fail(RS_ERR_INVALID, "va, vb and vout go together");
  KeyXform x;
  if (rs_status st = key_xform(plan, &x); st != RS_OK) return st;
  const uint32_t tile = merge_tile_keys(plan ? plan->tile : 0u, pairs);
  if (tile == 0) return fail(RS_ERR_UNSUPPORTED, "no merge tile shape %u", plan->tile);
  const size_t tiles = (size_t(n) + tile - 1) / tile;
  const size_t need = align_up((tiles + 1) * 4);
  if (!temp) {
    *temp_bytes = need;
    return RS_OK;
  }
  if (reinterpret_cast<uintptr_t>(temp) % kAlign) return fail(RS_ERR_INVALID, "temp is not 256-byte aligned");
  if (*temp_bytes < need) return fail(RS_ERR_TEMP_TOO_SMALL, "temp_bytes = %zu, need %zu", *temp_bytes, need);
  if ((na && !a) || (nb && !b) || (n && !out)) return fail(RS_ERR_INVALID, "NULL key buffer");
  if ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b) | reinterpret_cast<uintptr_t>(out) |
       reinterpret_cast<uintptr_t>(va) | reinterpret_cast<uintptr_t>(vb) | reinterpret_cast<uintptr_t>(vout)) & 3)
    return fail(RS_ERR_INVALID, "buffers must be 4-byte aligned");
  const void* ins[4] = {a, b, va, vb};
  const size_t in_n[4] = {size_t(na) * 4, size_t(nb) * 4, size_t(na) * 4, size_t(nb) * 4};
  for (const void* o : {static_cast<const void*>(out), static_cast<const void*>(vout)}) {
    for (int i = 0; i < 4; ++i)
      if (overlaps(o, size_t(n) * 4, ins[i], in_n[i])) return fail(RS_ERR_INVALID, "an output overlaps an input");
    if (overlaps(o, size_t(n) * 4, temp, need)) return fail(RS_ERR_INVALID, "an output overlaps temp");
  }
  if (pairs && overlaps(out, size_t(n) * 4, vout, size_t(n) * 4)) return fail(RS_ERR_INVALID, "out and vout overlap");
  if (h_part_offsets) part_offsets_host(n, num_parts, h_part_offsets);
  if (n == 0) return RS_OK;
  DeviceState* ds = nullptr;
  if (rs_status st = device_state(&ds); st != RS_OK) return st;
  MergeArgs m{a, b, va, vb, out, vout, uint32_t(na), uint32_t(nb), static_cast<uint32_t*>(temp), x, ds->err, tile};
  RS_CUDA(traced(T_MERGE, double(n), s, [&] { return launch_merge(m, s); }), "launch merge");
  return RS_OK;
}

rs_status rs_sort_u32_host(const uint32_t* h_keys_in, const uint32_t* h_vals_in, uint32_t* h_keys_out,
                           uint32_t* h_vals_out, uint64_t n, uint32_t num_parts, uint64_t* h_part_offsets,
                           const rs_plan* plan, void* temp, size_t* temp_bytes, rs_stream_t stream) {
  g_last_error.clear();
  const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const bool pairs = h_vals_in != nullptr;
  if (!temp_bytes) return fail(RS_ERR_INVALID, "temp_bytes is NULL");
  if (!pairs && h_vals_out) return fail(RS_ERR_INVALID, "h_vals_out given without h_vals_in");
  if (pairs && !h_vals_out) return fail(RS_ERR_INVALID, "h_vals_in given without h_vals_out");
  if (n >= (uint64_t(1) << 32)) return fail(RS_ERR_INVALID, "n = %llu: must be below 2^32", (unsigned long long)n);
  // device copies of the arrays first, then the device sort's own scratch
  const size_t nb = size_t(n) * 4, slot = align_up(nb);
  const int nbuf = pairs ? 4 : 2;
  size_t sort_bytes = 0;
  rs_status st = sort_impl(nullptr, nullptr, nullptr, nullptr, n, num_parts, nullptr, plan, nullptr, &sort_bytes, s,
                           pairs);
  if (st != RS_OK) return st;
  const size_t need = nbuf * slot + sort_bytes;
  if (!temp) {
    *temp_bytes = need;
    return RS_OK;
  }
  if (reinterpret_cast<uintptr_t>(temp) % kAlign) return fail(RS_ERR_INVALID, "temp is not 256-byte aligned");
  if (*temp_bytes < need) return fail(RS_ERR_TEMP_TOO_SMALL, "temp_bytes = %zu, need %zu", *temp_bytes, need);
  if (n > 0) {
    if (!h_keys_in || !h_keys_out) return fail(RS_ERR_INVALID, "NULL host key buffer");
    const void* ins[2] = {h_keys_in, h_vals_in};
    const void* outs[2] = {h_keys_out, h_vals_out};
    for (const void* o : outs)
      for (const void* i : ins)
        if (overlaps(o, nb, i, nb)) return fail(RS_ERR_INVALID, "a host output overlaps a host input");
    if (pairs && overlaps(h_keys_out, nb, h_vals_out, nb)) return fail(RS_ERR_INVALID, "h_keys_out and h_vals_out overlap");
  }
  unsigned char* t = static_cast<unsigned char*>(temp);
  uint32_t* d_kin = reinterpret_cast<uint32_t*>(t);
  uint32_t* d_kout = reinterpret_cast<uint32_t*>(t + slot);
  uint32_t* d_vin = pairs ? reinterpret_cast<uint32_t*>(t + 2 * slot) : nullptr;
  uint32_t* d_vout = pairs ? reinterpret_cast<uint32_t*>(t + 3 * slot) : nullptr;
  if (n == 0) {  // num_parts was checked by the size query above
    if (h_part_offsets) part_offsets_host(0, num_parts, h_part_offsets);
    return RS_OK;
  }
  RS_CUDA(traced(T_H2D, double(n), s,
                 [&] { return cudaMemcpyAsync(d_kin, h_keys_in, nb, cudaMemcpyHostToDevice, s); }),
          "cudaMemcpyAsync(keys to device)");
  if (pairs)
    RS_CUDA(traced(T_H2D, double(n), s,
                   [&] { return cudaMemcpyAsync(d_vin, h_vals_in, nb, cudaMemcpyHostToDevice, s); }),
            "cudaMemcpyAsync(values to device)");
  size_t sb = sort_bytes;
  st = sort_impl(d_kin, d_vin, d_kout, d_vout, n, num_parts, h_part_offsets, plan, t + nbuf * slot, &sb, s, pairs);
  if (st != RS_OK) return st;
  RS_CUDA(traced(T_D2H, double(n), s,
                 [&] { return cudaMemcpyAsync(h_keys_out, d_kout, nb, cudaMemcpyDeviceToHost, s); }),
          "cudaMemcpyAsync(keys to host)");
  if (pairs)
    RS_CUDA(traced(T_D2H, double(n), s,
                   [&] { return cudaMemcpyAsync(h_vals_out, d_vout, nb, cudaMemcpyDeviceToHost, s); }),
            "cudaMemcpyAsync(values to host)");
  return RS_OK;
}

rs_status rs_sort_u32_segmented(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out,
                                uint32_t* vals_out, const uint64_t* d_seg_offsets, const uint64_t* h_seg_offsets,
                                uint32_t num_segs, uint64_t total_n, uint32_t num_parts, uint64_t* d_part_offsets,
                                const rs_plan* plan, void* temp, size_t* temp_bytes, rs_stream_t stream) {
  g_last_error.clear();
  const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const bool pairs = vals_in != nullptr;
  if (!temp_bytes) return fail(RS_ERR_INVALID, "temp_bytes is NULL");
  if (!pairs && vals_out) return fail(RS_ERR_INVALID, "vals_out given without vals_in");
  if (pairs && !vals_out) return fail(RS_ERR_INVALID, "vals_in given without vals_out");
  if (num_parts < 1) return fail(RS_ERR_INVALID, "num_parts must be >= 1");
  if (num_segs > 0 && !h_seg_offsets) return fail(RS_ERR_INVALID, "h_seg_offsets is NULL");
  if (total_n >= (uint64_t(1) << 32)) return fail(RS_ERR_INVALID, "total_n must be below 2^32");
  uint64_t max_seg = 0;
  if (num_segs > 0) {
    if (h_seg_offsets[0] != 0 || h_seg_offsets[num_segs] != total_n)
      return fail(RS_ERR_INVALID, "segment offsets must start at 0 and end at total_n");
    for (uint32_t i = 0; i < num_segs; ++i) {
      if (h_seg_offsets[i + 1] < h_seg_offsets[i]) return fail(RS_ERR_INVALID, "segment offsets decrease at %u", i);
      const uint64_t m = h_seg_offsets[i + 1] - h_seg_offsets[i];
      if (m > max_seg) max_seg = m;
    }
  }
  const rs_plan eff = resolve_plan(pairs ? RS_ENTRY_SEGMENTED_PAIRS : RS_ENTRY_SEGMENTED,
                                   num_segs ? (total_n + num_segs - 1) / num_segs : 0, plan);
  if (eff.digit_bits && eff.digit_bits != 8) return fail(RS_ERR_UNSUPPORTED, "the segmented sort uses 8-bit digits");
  if (eff.tile > uint32_t(kSegShapes))
    return fail(RS_ERR_UNSUPPORTED, "the segmented sort has tile shapes 1 to %d (got %u)", kSegShapes, eff.tile);
  if (eff.mode > RS_MODE_MSD) return fail(RS_ERR_INVALID, "unknown mode %u", eff.mode);
  const int shape = eff.tile ? int(eff.tile) - 1 : kSegDefaultShape;
  // MSD (and automatic): every segment that fits one block is sorted there
  // (bucket, then local sort); LSD: only the smallest class is, larger
  // segments go through the tiled passes.
  const uint32_t small_max = eff.mode == RS_MODE_LSD ? seg_kernels()->tiny_max : seg_kernels()->small_max;
  KeyXform xf;
  if (rs_status st = key_xform(&eff, &xf); st != RS_OK) return st;
  if (needs_wide_status(total_n)) return fail(RS_ERR_UNSUPPORTED, "the segmented sort needs total_n < 2^30 - 2^16");
  (void)max_seg;
  const SegLayout L = make_seg_layout(0, num_segs, total_n, 4, pairs, shape);
  if (!temp) {
    *temp_bytes = L.end;
    return RS_OK;
  }
  if (reinterpret_cast<uintptr_t>(temp) % kAlign) return fail(RS_ERR_INVALID, "temp is not 256-byte aligned");
  if (*temp_bytes < L.end) return fail(RS_ERR_TEMP_TOO_SMALL, "temp_bytes = %zu, need %zu", *temp_bytes, L.end);
  if (total_n > 0 && (!keys_in || !keys_out || !d_seg_offsets))
    return fail(RS_ERR_INVALID, "NULL buffer");
  const size_t nb = size_t(total_n) * 4;
  if (overlaps(keys_out, nb, keys_in, nb) || overlaps(keys_out, nb, temp, L.end) ||
      (pairs && (overlaps(vals_out, nb, vals_in, nb) || overlaps(vals_out, nb, keys_out, nb) ||
                 overlaps(vals_out, nb, keys_in, nb) || overlaps(vals_out, nb, temp, L.end) ||
                 overlaps(keys_out, nb, vals_in, nb))))
    return fail(RS_ERR_INVALID, "an output overlaps another buffer");
  if (num_segs == 0) return RS_OK;
  DeviceState* ds = nullptr;
  rs_status st = device_state(&ds);
  if (st != RS_OK) return st;
  if (d_part_offsets) {
    const size_t cnt = size_t(num_segs) * (num_parts + 1);
    RS_CUDA(traced(T_SEGOFF, 0, s,
                   [&] {
                     seg_part_offsets_kernel<<<unsigned((cnt + 255) / 256), 256, 0, s>>>(d_seg_offsets, num_segs,
                                                                                         num_parts, d_part_offsets);
                     return cudaGetLastError();
                   }),
            "launch seg_part_offsets");
  }
  if (total_n == 0) return RS_OK;
  return run_segmented(L, static_cast<unsigned char*>(temp), keys_in, pairs ? vals_in : nullptr, keys_out,
                       pairs ? vals_out : nullptr, d_seg_offsets, num_segs, 4, xf, xf, ds, s, small_max);
}

rs_status rs_digit_histograms(const uint32_t* keys, uint64_t n, uint32_t digit_bits, uint32_t* d_hist,
                              uint32_t* d_bases, uint32_t* d_skip, rs_stream_t stream) {
  g_last_error.clear();
  const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (digit_bits != 8 && digit_bits != 11) return fail(RS_ERR_UNSUPPORTED, "digit_bits must be 8 or 11");
  if (n >= (uint64_t(1) << 32)) return fail(RS_ERR_INVALID, "n must be below 2^32");
  if (!d_hist) return fail(RS_ERR_INVALID, "d_hist is NULL");
  if (n > 0 && !keys) return fail(RS_ERR_INVALID, "keys is NULL");
  if (reinterpret_cast<uintptr_t>(keys) & 3) return fail(RS_ERR_INVALID, "keys must be 4-byte aligned");
  HistArgs ha{};
  ha.keys = keys;
  ha.n = uint32_t(n);
  ha.num_digits = 0;
  for (uint32_t sft = 0; sft < 32; sft += digit_bits) {
    ha.dig[ha.num_digits].shift = sft;
    ha.dig[ha.num_digits].width = (32 - sft) < digit_bits ? (32 - sft) : digit_bits;
    ++ha.num_digits;
  }
  ha.hist = d_hist;
  DeviceState* ds = nullptr;
  rs_status st = device_state(&ds);
  if (st != RS_OK) return st;
  const size_t bytes = size_t(ha.num_digits) * (size_t(1) << digit_bits) * 4;
  RS_CUDA(traced(T_CLEAR, 0, s, [&] { return cudaMemsetAsync(d_hist, 0, bytes, s); }), "cudaMemsetAsync(hist)");
  if (n > 0) {
    const size_t work = (size_t(n) + 4095) / 4096;
    unsigned grid = unsigned(ds->num_sms) * (hist_kernel(int(digit_bits))->threads >= 1024 ? 1 : 2);
    if (work < grid) grid = unsigned(work);
    RS_CUDA(traced(T_HIST, double(n), s, [&] { return hist_kernel(int(digit_bits))->launch(ha, grid, s); }),
            "launch upfront_hist");
  }
  if (d_bases || d_skip) {
    uint32_t* b = d_bases;
    if (!b) return fail(RS_ERR_INVALID, "d_skip needs d_bases");
    ScanArgs sa{d_hist, b, d_skip, uint32_t(n)};
    RS_CUDA(traced(T_SCAN, 0, s, [&] { return scan_kernel(int(digit_bits))->launch(sa, unsigned(ha.num_digits), s); }),
            "launch digit_scan");
  }
  return RS_OK;
}

rs_status rs_radix_pass(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out, uint32_t* vals_out,
                        uint64_t n, uint32_t shift, uint32_t width, void* temp, size_t* temp_bytes,
                        rs_stream_t stream) {
  g_last_error.clear();
  const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  rs_status st = check_common(keys_in, keys_out, n, temp, temp_bytes);
  if (st != RS_OK) return st;
  if (width < 1 || width > 11 || shift + width > 32) return fail(RS_ERR_INVALID, "bad digit (shift %u, width %u)", shift, width);
  const bool pairs = vals_in != nullptr;
  if (pairs != (vals_out != nullptr)) return fail(RS_ERR_INVALID, "vals_in and vals_out must both be given or both NULL");
  SortPlan p;
  p.R = width > 8 ? 11 : 8;
  p.nd = 1;
  p.dig[0].shift = shift;
  p.dig[0].width = width;
  st = pick_kernel(p.R, 0, pairs, needs_wide_status(n), &p.k);
  if (st != RS_OK) return st;
  p.num_tiles = (n + p.k->tile - 1) / p.k->tile;
  const Layout L = make_layout(p, n, pairs);
  if (!temp) {
    *temp_bytes = L.total;
    return RS_OK;
  }
  if (*temp_bytes < L.total) return fail(RS_ERR_TEMP_TOO_SMALL, "temp_bytes = %zu, need %zu", *temp_bytes, L.total);
  const size_t nb = size_t(n) * 4;
  if (overlaps(keys_out, nb, keys_in, nb) || overlaps(keys_out, nb, temp, L.total) ||
      (pairs && (overlaps(vals_out, nb, vals_in, nb) || overlaps(vals_out, nb, keys_out, nb) ||
                 overlaps(vals_out, nb, keys_in, nb) || overlaps(keys_out, nb, vals_in, nb) ||
                 overlaps(vals_out, nb, temp, L.total))))
    return fail(RS_ERR_INVALID, "an output overlaps another buffer");
  if (n == 0) return RS_OK;
  DeviceState* ds = nullptr;
  st = device_state(&ds);
  if (st != RS_OK) return st;
  return run_lsd(p, L, keys_in, vals_in, keys_out, vals_out, uint32_t(n), static_cast<unsigned char*>(temp), true,
                 ds, s);
}

rs_status rs_sample_overlap(const uint32_t* keys, uint64_t n, uint32_t key_kind, uint32_t bits, uint32_t sample,
                            uint32_t cells, uint32_t max_problem, uint32_t* d_buckets, uint32_t* h_out,
                            rs_stream_t stream) {
  g_last_error.clear();
  if (!h_out) return fail(RS_ERR_INVALID, "h_out is NULL");
  if (n > 0 && !keys) return fail(RS_ERR_INVALID, "NULL keys");
  if (reinterpret_cast<uintptr_t>(keys) & 3) return fail(RS_ERR_INVALID, "keys must be 4-byte aligned");
  if (bits < 1 || bits > 32) return fail(RS_ERR_INVALID, "bits must be 1..32 (got %u)", bits);
  if (sample < 1 || sample > 1024) return fail(RS_ERR_INVALID, "sample must be 1..1024 (got %u)", sample);
  if (cells < 1 || cells > 1024) return fail(RS_ERR_INVALID, "cells must be 1..1024 (got %u)", cells);
  const rs_plan kind_only = {0, 0, 0, key_kind};
  KeyXform xf;
  if (rs_status st = key_xform(&kind_only, &xf); st != RS_OK) return st;
  if (n == 0) {
    h_out[0] = h_out[1] = h_out[2] = h_out[3] = 0;
    return RS_OK;
  }
  DeviceState* ds = nullptr;
  if (rs_status st = device_state(&ds); st != RS_OK) return st;
  const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> lock(g_select_mu);
  uint32_t* d_out = nullptr;
  RS_CUDA(cudaGetSymbolAddress(reinterpret_cast<void**>(&d_out), g_select_out), "cudaGetSymbolAddress(select)");
  SelectArgs a{keys, n, xf, bits, sample, cells, max_problem, d_out, d_buckets};
  RS_CUDA(traced(T_SELECT, double(n), s, [&] { return launch_select(a, s); }), "launch select");
  RS_CUDA(cudaMemcpyAsync(h_out, d_out, 4 * sizeof(uint32_t), cudaMemcpyDeviceToHost, s), "read selection");
  RS_CUDA(cudaStreamSynchronize(s), "cudaStreamSynchronize");
  return RS_OK;
}

rs_status rs_choose_plan(const uint32_t* keys, uint64_t n, const rs_plan* base, rs_plan* out, uint32_t* h_stats,
                         rs_stream_t stream) {
  g_last_error.clear();
  if (!out) return fail(RS_ERR_INVALID, "out is NULL");
  const rs_plan eff = resolve_plan(RS_ENTRY_SORT_U32, n, base);
  uint32_t st4[4] = {0, 0, 0, 0};
  if (rs_status st = rs_sample_overlap(keys, n, eff.key_kind, kSelectBits, kSelectSample, kSelectCells,
                                       kSelectMaxProblem, nullptr, st4, stream);
      st != RS_OK)
    return st;
  *out = eff;
  if (st4[1] && eff.mode == RS_MODE_MSD) out->mode = RS_MODE_LSD;  // clustered: no bucketing plan
  if (h_stats)
    for (int i = 0; i < 4; ++i) h_stats[i] = st4[i];
  return RS_OK;
}

rs_status rs_set_default_plan(uint32_t entry, uint32_t size_class, const rs_plan* plan) {
  g_last_error.clear();
  if (entry >= uint32_t(kPlanEntries)) return fail(RS_ERR_INVALID, "unknown entry %u", entry);
  if (size_class >= uint32_t(kSizeClasses)) return fail(RS_ERR_INVALID, "size class %u above 32", size_class);
  if (plan) {
    if (plan->key_kind != RS_KEY_U32) return fail(RS_ERR_INVALID, "a default plan does not set key_kind");
    if (plan->mode > RS_MODE_MSD) return fail(RS_ERR_INVALID, "unknown mode %u", plan->mode);
    if (plan->digit_bits && plan->digit_bits != 8 && plan->digit_bits != 11)
      return fail(RS_ERR_UNSUPPORTED, "digit_bits must be 0, 8 or 11 (got %u)", plan->digit_bits);
  }
  std::lock_guard<std::mutex> lock(g_plan_mu);
  g_plan_set[entry][size_class] = plan != nullptr;
  g_plan_table[entry][size_class] = plan ? *plan : rs_plan{0, 0, 0, 0};
  return RS_OK;
}

rs_status rs_get_default_plan(uint32_t entry, uint32_t size_class, rs_plan* out, int* is_set) {
  g_last_error.clear();
  if (!out || !is_set) return fail(RS_ERR_INVALID, "NULL output");
  if (entry >= uint32_t(kPlanEntries)) return fail(RS_ERR_INVALID, "unknown entry %u", entry);
  if (size_class >= uint32_t(kSizeClasses)) return fail(RS_ERR_INVALID, "size class %u above 32", size_class);
  std::lock_guard<std::mutex> lock(g_plan_mu);
  *is_set = g_plan_set[entry][size_class] ? 1 : 0;
  *out = g_plan_table[entry][size_class];
  return RS_OK;
}

const char* rs_last_error(void) { return g_last_error.c_str(); }

rs_status rs_check_device_error(rs_stream_t stream) {
  g_last_error.clear();
  DeviceState* ds = nullptr;
  rs_status st = device_state(&ds);
  if (st != RS_OK) return st;
  const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // One thread takes the word (atomic exchange with zero) after the stream's
  // earlier work; the host then reads what it took.  Serialised per device so
  // that two checking threads do not share the copy word.
  uint32_t word = 0;
  {
    std::lock_guard<std::mutex> lock(g_err_mu);
    take_error_kernel<<<1, 1, 0, s>>>(ds->err, ds->err_taken);
    RS_CUDA(cudaGetLastError(), "launch take_error");
    RS_CUDA(cudaMemcpyAsync(&word, ds->err_taken, sizeof(word), cudaMemcpyDeviceToHost, s), "read device error word");
    RS_CUDA(cudaStreamSynchronize(s), "cudaStreamSynchronize");
  }
  if (word) {
    if (word & kErrTimeout) return fail(RS_ERR_TIMEOUT, "a bounded device-side wait gave up (error word 0x%x)", word);
    return fail(RS_ERR_CUDA, "a device-side output index check fired (error word 0x%x)", word);
  }
  return RS_OK;
}

rs_status rs_peek_device_error_async(uint32_t* h_word, rs_stream_t stream) {
  g_last_error.clear();
  if (!h_word) return fail(RS_ERR_INVALID, "h_word is NULL");
  DeviceState* ds = nullptr;
  rs_status st = device_state(&ds);
  if (st != RS_OK) return st;
  RS_CUDA(cudaMemcpyAsync(h_word, ds->err, sizeof(uint32_t), cudaMemcpyDeviceToHost,
                          reinterpret_cast<cudaStream_t>(stream)),
          "copy device error word");
  return RS_OK;
}

rs_status rs_trace_enable(int on) {
  g_last_error.clear();
  std::lock_guard<std::mutex> lock(g_trace_mu);
  g_trace_on = on != 0;
  return RS_OK;
}

rs_status rs_trace_read(rs_trace_entry* out, uint32_t capacity, uint32_t* count) {
  g_last_error.clear();
  if (!count || (capacity > 0 && !out)) return fail(RS_ERR_INVALID, "NULL output");
  std::lock_guard<std::mutex> lock(g_trace_mu);
  uint32_t launches[T_KINDS] = {};
  double ms[T_KINDS] = {}, keys[T_KINDS] = {};
  rs_status st = RS_OK;
  for (TraceRec& r : g_trace) {
    float t = 0.f;
    cudaError_t e = cudaEventSynchronize(r.b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.a, r.b);
    if (e != cudaSuccess && st == RS_OK) st = cuda_fail(e, "trace event");
    ++launches[r.kind];
    ms[r.kind] += t;
    keys[r.kind] += r.keys;
    g_event_pool.push_back(r.a);
    g_event_pool.push_back(r.b);
  }
  g_trace.clear();
  uint32_t c = 0;
  for (int k = 0; k < T_KINDS; ++k) {
    if (!launches[k]) continue;
    if (c < capacity) {
      std::memset(&out[c], 0, sizeof(out[c]));
      std::snprintf(out[c].name, sizeof(out[c].name), "%s", kTraceNames[k]);
      out[c].launches = launches[k];
      out[c].total_ms = ms[k];
      out[c].keys = keys[k];
    }
    ++c;
  }
  *count = c < capacity ? c : capacity;
  return st;
}

rs_status rs_selftest_wait_timeout(void* temp, size_t temp_bytes, rs_stream_t stream) {
  g_last_error.clear();
  if (!temp || temp_bytes < 4096) return fail(RS_ERR_INVALID, "the self-test needs 4096 bytes of temp");
  if (reinterpret_cast<uintptr_t>(temp) % kAlign) return fail(RS_ERR_INVALID, "temp is not 256-byte aligned");
  DeviceState* ds = nullptr;
  rs_status st = device_state(&ds);
  if (st != RS_OK) return st;
  const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  RS_CUDA(cudaMemsetAsync(temp, 0, 4096, s), "cudaMemsetAsync(self-test)");
  RS_CUDA(launch_lookback_timeout(static_cast<const uint32_t*>(temp), ds->err, s), "launch self-test");
  return RS_OK;
}

uint32_t rs_version(void) { return kVersion; }

}  // extern "C"
