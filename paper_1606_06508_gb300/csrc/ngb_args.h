// ngb_args.h -- the host-side argument checks of the forward, backward and
// no-alloc entry points of include/normgb.h, in one place.  Plain C++ with no
// CUDA dependency: the library compiles it into api.cu and noalloc.cu, and the
// CPU tests compile the same header into a host harness, so that a test
// stand-in accepts and rejects exactly what the library does.
//
// Element arrays of a ragged batch (dim == 0) may be NULL: a batch whose
// vectors are all empty has no elements, and allocators commonly hand out a
// NULL address for a zero-byte buffer.  Nothing decides on the host whether
// the offsets describe such a batch (they live in device memory), so a ragged
// call with a NULL element array sets `no_elements`; the kernels then treat
// every vector of positive length as having bad offsets (skipped, reported
// through the plan's status word) and never form an address from the NULL
// pointer.  Zero-length vectors are finished as usual (norm +0).
#pragma once
#include <stdint.h>

#include "normgb.h"

namespace ngb {

struct ArgCheck {
  ngb_status status;    // NGB_OK, or the status the entry point returns
  const char* message;  // reason for a non-OK status ("" otherwise)
  bool no_elements;     // ragged call with a NULL element array (see above)
};

inline ArgCheck arg_ok(bool no_elements) { return ArgCheck{NGB_OK, "", no_elements}; }
inline ArgCheck arg_fail(ngb_status s, const char* m) { return ArgCheck{s, m, false}; }

// Checks shared by the forward and backward calls: sizes, flags, offsets.
inline ArgCheck check_shape(int64_t count, int32_t dim, const void* offsets, uint32_t flags) {
  if (count < 0) return arg_fail(NGB_ERR_INVALID_ARG, "count < 0");
  if (dim < 0) return arg_fail(NGB_ERR_INVALID_ARG, "dim < 0");
  if (dim > NGB_MAX_LEN) return arg_fail(NGB_ERR_UNSUPPORTED, "dim > NGB_MAX_LEN");
  if (flags & ~(uint32_t)(NGB_VECTOR_SEMANTICS | NGB_VALIDATE_OFFSETS))
    return arg_fail(NGB_ERR_INVALID_ARG, "unknown flag");
  if (dim > 0 && offsets) return arg_fail(NGB_ERR_INVALID_ARG, "offsets given for a dense batch (dim > 0)");
  if (dim == 0 && !offsets) return arg_fail(NGB_ERR_INVALID_ARG, "ragged batch (dim == 0) needs offsets");
  if (dim == 0 && count > INT32_MAX) return arg_fail(NGB_ERR_UNSUPPORTED, "ragged count >= 2^31");
  return arg_ok(false);
}

// normalize_f32 / normalize_f64.  y, norm, saved_h and saved_code are
// nullable (y == NULL computes norms only).  A dense batch (dim > 0) with
// count > 0 has count * dim > 0 elements, so x is required there.
inline ArgCheck check_forward(const void* x, int64_t count, int32_t dim, const void* offsets, uint32_t flags) {
  const ArgCheck a = check_shape(count, dim, offsets, flags);
  if (a.status != NGB_OK) return a;
  if (count > 0 && dim > 0 && !x) return arg_fail(NGB_ERR_INVALID_ARG, "x is NULL");
  return arg_ok(dim == 0 && !x);
}

// normalize_backward_f32 / _f64.  saved_h and saved_code hold one entry per
// vector and are required whenever count > 0; y, g and grad are required for
// a dense batch and may be NULL for a ragged one (no_elements).
inline ArgCheck check_backward(const void* y, const void* g, const void* saved_h, const void* saved_code,
                               const void* grad, int64_t count, int32_t dim, const void* offsets, uint32_t flags) {
  const ArgCheck a = check_shape(count, dim, offsets, flags);
  if (a.status != NGB_OK) return a;
  if (count > 0 && (!saved_h || !saved_code))
    return arg_fail(NGB_ERR_INVALID_ARG, "saved_h and saved_code are required");
  if (count > 0 && dim > 0 && (!y || !g || !grad))
    return arg_fail(NGB_ERR_INVALID_ARG, "y, g and grad are required for a dense batch");
  return arg_ok(dim == 0 && (!y || !g || !grad));
}

// normalize_ragged_f32_noalloc: a ragged forward with a fixed maximum count.
inline ArgCheck check_noalloc(const void* x, int64_t count, const void* offsets, uint32_t flags) {
  if (count < 0) return arg_fail(NGB_ERR_INVALID_ARG, "count < 0");
  if (count > NGB_NOALLOC_MAX_COUNT)
    return arg_fail(NGB_ERR_UNSUPPORTED,
                    "count exceeds NGB_NOALLOC_MAX_COUNT (262144); use a plan for larger batches");
  if (flags & ~(uint32_t)NGB_VALIDATE_OFFSETS) return arg_fail(NGB_ERR_INVALID_ARG, "unknown flag");
  if (count > 0 && !offsets) return arg_fail(NGB_ERR_INVALID_ARG, "offsets are required");
  return arg_ok(!x);
}

// The element capacity handed to the classifier: the caller's capacity
// (> 0: ends past it are bad offsets; 0: unknown), or -1 when the batch has
// no element array, so that every vector of positive length is bad.
inline int64_t classifier_capacity(int64_t capacity, bool no_elements) { return no_elements ? -1 : capacity; }

}  // namespace ngb
