// noalloc.cu -- normalize_ragged_f32_noalloc: the ragged binary32 forward
// pass without any device allocation.  The classifier's work lists and
// counters, which ngb_plan_create would otherwise cudaMalloc, live in one
// file-scope __device__ array of fixed size that every device loading the
// library keeps until the process exits.
#include <mutex>
#include <string>

#include "normgb.h"
#include "ngb_args.h"
#include "ngb_internal.h"

namespace {

// The counters and status words (ngb::SCRATCH_HEADER_WORDS) followed by the
// three binary32 work lists of NGB_NOALLOC_MAX_COUNT vector indices:
// (16 + 3 * 262144) * 4 bytes, about 3 MiB.
constexpr int64_t kScratchWords =
    ngb::SCRATCH_HEADER_WORDS + ngb::ragged_lists(4) * (int64_t)NGB_NOALLOC_MAX_COUNT;
__device__ __align__(256) int32_t g_noalloc_scratch[kScratchWords];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
int32_t* g_scratch_addr[kMaxDevices] = {nullptr};  // device address of g_noalloc_scratch, per device

// Host code cannot use g_noalloc_scratch as a device address: its name in host
// code refers to a host-side shadow.  The device address is looked up once per
// device, with that device current, and kept.
cudaError_t scratch_for_current_device(int32_t** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<int32_t*>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" ngb_status normalize_ragged_f32_noalloc(const float* x, float* y, float* norm, float* saved_h,
                                                   int8_t* saved_code, int64_t count, const int64_t* offsets,
                                                   uint32_t flags, ngb_stream_t stream) {
  ngb::set_last_error("");
  const ngb::ArgCheck a = ngb::check_noalloc(x, count, offsets, flags);
  if (a.status != NGB_OK) return ngb::set_last_error(a.message), a.status;
  if (count == 0) return NGB_OK;
  int32_t* base = nullptr;
  cudaError_t e = scratch_for_current_device(&base);
  if (e != cudaSuccess)
    return ngb::set_last_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e)), NGB_ERR_CUDA;
  // Same layout as a plan's buffer (ngb::ragged_scratch); launch_ragged
  // clears the counts and tickets on the stream before use.
  const ngb::RaggedScratch sc = ngb::ragged_scratch(base);
  ngb::RaggedMapping map{8, 8192, 256, 0};
  map.grid_blocks = ngb::ragged_full_wave<float>(map, false);
  e = ngb::launch_ragged<float>(x, y, norm, saved_h, saved_code, nullptr, nullptr, nullptr, nullptr, offsets, count,
                                ngb::classifier_capacity(0, a.no_elements), (flags & NGB_VALIDATE_OFFSETS) != 0, map, sc, false,
                                reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return ngb::set_last_error(std::string("launch: ") + cudaGetErrorString(e)), NGB_ERR_CUDA;
  return NGB_OK;
}
