// fixed_f32.cu -- binary32 instantiation of the dense-batch kernels.
#include "kernels_fixed.cuh"

namespace ngb {
template <>
cudaError_t launch_fixed_forward<float>(const float* x, float* y, float* norm, float* h, int8_t* code, int64_t count,
                                        int dim, bool quat_zero, cudaStream_t s) {
  return launch_fixed_forward_impl<float>(x, y, VecOut<float>{norm, h, code}, count, dim, quat_zero, s);
}
template <>
cudaError_t launch_fixed_backward<float>(const float* y, const float* g, const float* h, const int8_t* c,
                                         float* grad, int64_t count, int dim, cudaStream_t s) {
  return launch_fixed_backward_impl<float>(y, g, h, c, grad, count, dim, s);
}
}  // namespace ngb
