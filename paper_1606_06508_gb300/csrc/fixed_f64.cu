// fixed_f64.cu -- binary64 instantiation of the dense-batch kernels.
#include "kernels_fixed.cuh"

namespace ngb {
template <>
cudaError_t launch_fixed_forward<double>(const double* x, double* y, double* norm, double* h, int8_t* code, int64_t count,
                                        int dim, bool quat_zero, cudaStream_t s) {
  return launch_fixed_forward_impl<double>(x, y, VecOut<double>{norm, h, code}, count, dim, quat_zero, s);
}
template <>
cudaError_t launch_fixed_backward<double>(const double* y, const double* g, const double* h, const int8_t* c,
                                         double* grad, int64_t count, int dim, cudaStream_t s) {
  return launch_fixed_backward_impl<double>(y, g, h, c, grad, count, dim, s);
}
}  // namespace ngb
