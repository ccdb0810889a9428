// ragged_f64.cu -- binary64 instantiation of the ragged-batch kernels.
#include "kernels_ragged.cuh"

namespace ngb {
template <>
cudaError_t launch_ragged<double>(const double* x, double* y, double* norm, double* saved_h, int8_t* saved_code,
                                 const double* g, const double* h_in, const int8_t* code_in, double* grad,
                                 const int64_t* offsets, int64_t count, int64_t capacity, bool validate,
                                 const RaggedMapping& map, const RaggedScratch& sc, bool backward, cudaStream_t s) {
  return launch_ragged_impl<double>(x, y, norm, saved_h, saved_code, g, h_in, code_in, grad, offsets, count,
                                   capacity, validate, map, sc, backward, s);
}
template <>
int ragged_full_wave<double>(const RaggedMapping& map, bool backward) {
  // the backward lists run one full wave per kernel
  return backward ? 0 : full_wave_dispatch<double>(map);
}
}  // namespace ngb
