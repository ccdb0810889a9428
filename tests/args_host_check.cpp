// The library's argument checks (paper_1606_06508_gb300/csrc/ngb_args.h)
// compiled for the host as a small shared library, so that CPU tests can ask
// whether the C ABI accepts a call: the test stand-in for the library
// (tests/test_guarded_host.py) applies exactly these checks before answering
// through the oracle.
#include "ngb_args.h"

extern "C" {

// Each returns the ngb_status of the check and sets *no_elements.
int host_check_forward(const void* x, int64_t count, int32_t dim, const void* offsets, uint32_t flags,
                       int* no_elements) {
  const ngb::ArgCheck a = ngb::check_forward(x, count, dim, offsets, flags);
  *no_elements = a.no_elements ? 1 : 0;
  return a.status;
}

int host_check_backward(const void* y, const void* g, const void* saved_h, const void* saved_code, const void* grad,
                        int64_t count, int32_t dim, const void* offsets, uint32_t flags, int* no_elements) {
  const ngb::ArgCheck a = ngb::check_backward(y, g, saved_h, saved_code, grad, count, dim, offsets, flags);
  *no_elements = a.no_elements ? 1 : 0;
  return a.status;
}

int host_check_noalloc(const void* x, int64_t count, const void* offsets, uint32_t flags, int* no_elements) {
  const ngb::ArgCheck a = ngb::check_noalloc(x, count, offsets, flags);
  *no_elements = a.no_elements ? 1 : 0;
  return a.status;
}

}  // extern "C"
