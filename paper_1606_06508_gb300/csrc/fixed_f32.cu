// fixed_f32.cu -- binary32 instantiation of the dense-batch kernels, and the
// bulk-copy quaternion kernel (ngb_bulk.cuh).
#include <cstdlib>
#include <mutex>

#include "kernels_fixed.cuh"
#include "ngb_bulk.cuh"

namespace ngb {

bool quat_bulk_enabled() {
  static const bool on = [] {
    const char* v = std::getenv("NGB_QUAT_BULK");
    return v && v[0] == '1' && v[1] == 0;
  }();
  return on;
}

cudaError_t quat_bulk_state(uint32_t* state) {
  unsigned v = 0;
  const cudaError_t e = cudaMemcpyFromSymbol(&v, g_bulk_state, sizeof(v));
  *state = v;
  return e;
}

static bool device_memory(const void* p) {
  if (!p) return true;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice;
}

cudaError_t launch_quat_bulk(const float* x, float* y, const VecOut<float>& out, int64_t count, bool quat_zero,
                             cudaStream_t s) {
  if (!aligned16(x) || !aligned16(y) || !device_memory(x) || !device_memory(y)) return cudaErrorNotSupported;
  static std::once_flag attr_once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(attr_once, [] {
    attr_err = cudaFuncSetAttribute(k_quat_bulk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BULK_SMEM);
  });
  if (attr_err != cudaSuccess) return attr_err;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_quat_bulk, BULK_THREADS, BULK_SMEM);
  if (per_sm < 1) per_sm = 1;
  const int64_t tiles = (count + BULK_TILE - 1) / BULK_TILE;
  const int64_t wave = (int64_t)device_sm_count() * per_sm;
  const int grid = (int)(tiles < wave ? tiles : wave);
  k_quat_bulk<<<grid, BULK_THREADS, BULK_SMEM, s>>>(x, y, out, count, quat_zero ? 1 : 0);
  return cudaGetLastError();
}

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
