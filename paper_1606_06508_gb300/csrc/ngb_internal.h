// ngb_internal.h -- host-side declarations shared by the translation units of
// the library (launchers, device properties, the ragged plan).  Not installed.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

namespace ngb {

template <typename T> struct VecOut;

// Multiprocessor count of the current device (cached per device).
int device_sm_count();

// Sets the message returned by ngb_last_error() on this thread.
void set_last_error(const std::string& msg);

// Dense [count][dim] batches.
template <typename T>
cudaError_t launch_fixed_forward(const T* x, T* y, T* norm, T* saved_h, int8_t* saved_code, int64_t count,
                                 int dim, bool quat_zero, cudaStream_t s);
template <typename T>
cudaError_t launch_fixed_backward(const T* y, const T* g, const T* h, const int8_t* c, T* grad, int64_t count,
                                  int dim, cudaStream_t s);

// binary32 quaternions through bulk copies into shared memory (ngb_bulk.cuh;
// fixed_f32.cu).  Returns cudaErrorNotSupported, launching nothing, unless x
// and y (when given) are 16-byte aligned device memory.  Taken instead of
// k_small_vec16 only when quat_bulk_enabled(): the environment variable
// NGB_QUAT_BULK is "1" when the library first asks (it measured slower).
cudaError_t launch_quat_bulk(const float* x, float* y, const VecOut<float>& out, int64_t count, bool quat_zero,
                             cudaStream_t s);
bool quat_bulk_enabled();
// The bulk path's state word on the current device (see ngb_quat_bulk_state).
cudaError_t quat_bulk_state(uint32_t* state);

// Ragged batches: bucket lists produced by the classifier, consumed by one
// persistent kernel.
struct RaggedMapping {
  int thread_max;     // n <= thread_max: one thread per vector (4 .. 16)
  int warp_max;       // thread_max < n <= warp_max: one warp per vector, streamed
  int block_threads;  // n > warp_max: one block of this many threads per vector (128 or 256)
  int grid_blocks;    // persistent grid size; 0 = one full wave
};

// The work lists of a ragged call, by length class: block items, warp items,
// thread items, and (binary64) the items of groups of 8 and of 16 lanes.
enum RaggedList { LIST_BLOCK = 0, LIST_WARP = 1, LIST_THREAD = 2, LIST_GROUP8 = 3, LIST_GROUP16 = 4, NLISTS = 5 };

// Words of the scratch header: counts[NLISTS], tickets[NLISTS], status, then
// padding to 16 words; the lists follow.
constexpr int SCRATCH_HEADER_WORDS = 16;

struct RaggedScratch {
  int32_t* items;    // list k at items[k * count], for the lists the dtype uses
  int32_t* counts;   // [NLISTS] items per list (filled by the classifier)
  int32_t* tickets;  // [NLISTS] work counters of the persistent kernel; adjacent to counts
  int32_t* status;   // bit 0: a vector with bad offsets was skipped
};

// Lists a dtype uses: binary32 has no group lists (the first three lists),
// binary64 all five.
constexpr int ragged_lists(int dtype_bytes) { return dtype_bytes == 8 ? NLISTS : 3; }

// RaggedScratch over a buffer of SCRATCH_HEADER_WORDS + lists * count words.
inline RaggedScratch ragged_scratch(int32_t* buf) {
  RaggedScratch sc;
  sc.counts = buf;
  sc.tickets = buf + NLISTS;
  sc.status = buf + 2 * NLISTS;
  sc.items = buf + SCRATCH_HEADER_WORDS;
  return sc;
}

template <typename T>
cudaError_t launch_ragged(const T* x, T* y, T* norm, T* saved_h, int8_t* saved_code, const T* g_or_null,
                          const T* h_in, const int8_t* code_in, T* grad, const int64_t* offsets, int64_t count,
                          int64_t capacity, bool validate, const RaggedMapping& map, const RaggedScratch& sc,
                          bool backward, cudaStream_t s);

// Grid of one full wave of the persistent ragged kernel for this mapping.
template <typename T>
int ragged_full_wave(const RaggedMapping& map, bool backward);

// Measurement aids and extra entry points.
cudaError_t launch_copy(void* dst, const void* src, int64_t bytes, cudaStream_t s);
cudaError_t launch_fp64_probe(double* out, int blocks, int iters, cudaStream_t s);
template <typename T>
cudaError_t launch_quotient3(const T* x, T* y, T* norm, int64_t count, int alg, cudaStream_t s);
template <typename T>
cudaError_t launch_naive(const T* x, T* y, int64_t count, int dim, cudaStream_t s);
template <typename T>
cudaError_t launch_rotation(const T* q, T* R, T* norm, int64_t count, cudaStream_t s);

}  // namespace ngb
