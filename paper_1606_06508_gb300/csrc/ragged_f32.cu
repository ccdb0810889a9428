// ragged_f32.cu -- binary32 instantiation of the ragged-batch kernels.
#include "kernels_ragged.cuh"

namespace ngb {
template <>
cudaError_t launch_ragged<float>(const float* x, float* y, float* norm, float* saved_h, int8_t* saved_code,
                                 const float* g, const float* h_in, const int8_t* code_in, float* grad,
                                 const int64_t* offsets, int64_t count, int64_t capacity, bool validate,
                                 const RaggedMapping& map, const RaggedScratch& sc, bool backward, cudaStream_t s) {
  return launch_ragged_impl<float>(x, y, norm, saved_h, saved_code, g, h_in, code_in, grad, offsets, count,
                                   capacity, validate, map, sc, backward, s);
}
template <>
int ragged_full_wave<float>(const RaggedMapping& map, bool backward) {
  // the backward lists run one full wave per kernel
  return backward ? 0 : full_wave_dispatch<float>(map);
}
}  // namespace ngb
