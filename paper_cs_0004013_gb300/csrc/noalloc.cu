// rs_sort_u32_noalloc: the keys-only sort for callers that cannot allocate
// device memory.
//
// The regular entry points take their scratch space from the caller (temp,
// temp_bytes), which the caller usually gets from cudaMalloc or from an
// allocator such as PyTorch's.  Some callers have neither: code embedded in
// a host program that owns every device allocation and hands out no
// allocator, code on a latency-critical path where cudaMalloc (which can
// synchronise the whole device) is not acceptable, and code that must not
// be able to fail with out-of-memory once it has started.  For them this
// entry point keeps its scratch in a fixed array that lives in the
// library's own device memory and is held until the process exits.  With
// CUDA's lazy module loading (the default), the module holding the array is
// loaded, and the array reserved, by the first call on each device (its
// cudaGetSymbolAddress); that first call can therefore still fail for lack
// of device memory.  Callers that must not fail later make it during set-up:
// a call with n = 0 does the set-up and sorts nothing.
//
// The array is sized for at most RS_NOALLOC_MAX_KEYS keys (about 4.5 MiB).
// Every call on a device uses the same array, and the array keeps whatever
// the last call left in it; the sort clears the parts that must start at
// zero (tile tickets, histograms, chained-scan status words) on every call.
// Two calls whose work overlaps on the GPU (for instance on two streams)
// race on the array and give wrong results: serialise them.
#include <cstdio>
#include <mutex>

#include <cuda_runtime.h>

#include "rs_internal.h"
#include "rsort.h"

namespace {

constexpr int kMaxDevices = 64;
// Scratch of the sort pinned below at RS_NOALLOC_MAX_KEYS keys: 4 MiB for the
// alternate key buffer plus the control block, histograms, bases and status
// words (under 100 KiB); checked against the sort's own size query.
constexpr size_t kScratchBytes = (size_t(4) << 20) + (size_t(512) << 10);
// 8-bit digits, 1024 x 16 tiles (shape index 3, given as tile = 4).
constexpr rs_plan kPlan = {8, RS_MODE_LSD, 4, 0};

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Looks up, once per device and with that device current, the device
// address of the scratch array (the host-side symbol is only a stand-in
// and must never be passed to a kernel).
rs_status scratch_for_current_device(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    rs::set_last_error(RS_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    return RS_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    rs::set_last_error(RS_ERR_UNSUPPORTED, "device index %d out of range", dev);
    return RS_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      rs::set_last_error(RS_ERR_CUDA, "cudaGetSymbolAddress(no-alloc scratch): %s", cudaGetErrorString(e));
      return RS_ERR_CUDA;
    }
    size_t need = 0;
    const rs_status st = rs_sort_u32(nullptr, nullptr, RS_NOALLOC_MAX_KEYS, 1, nullptr, &kPlan, nullptr, &need,
                                     nullptr);
    if (st != RS_OK) return st;
    if (need > kScratchBytes) {
      rs::set_last_error(RS_ERR_UNSUPPORTED, "no-alloc scratch holds %zu bytes but the sort needs %zu",
                         kScratchBytes, need);
      return RS_ERR_UNSUPPORTED;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return RS_OK;
}

}  // namespace

extern "C" rs_status rs_sort_u32_noalloc(const uint32_t* keys_in, uint32_t* keys_out, uint64_t n,
                                         uint32_t num_parts, uint64_t* h_part_offsets, rs_stream_t stream) {
  if (n > RS_NOALLOC_MAX_KEYS) {
    rs::set_last_error(RS_ERR_INVALID, "n = %llu exceeds the no-alloc limit of %u keys (use rs_sort_u32 with temp)",
                       (unsigned long long)n, unsigned(RS_NOALLOC_MAX_KEYS));
    return RS_ERR_INVALID;
  }
  void* scratch = nullptr;
  const rs_status st = scratch_for_current_device(&scratch);
  if (st != RS_OK) return st;
  size_t bytes = kScratchBytes;
  return rs_sort_u32(keys_in, keys_out, n, num_parts, h_part_offsets, &kPlan, scratch, &bytes, stream);
}
