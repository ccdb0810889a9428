// extras.cu -- device properties, the quaternion-to-rotation-matrix kernel and
// two measurement aids (a plain copy and the unscaled "naive" normalization).
#include <mutex>

#include "ngb_internal.h"
#include "ngb_rowpath.cuh"
#include "ngb_quotient.cuh"

namespace ngb {

int device_sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  if (cached[dev] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 152;
    cached[dev] = v;
  }
  return cached[dev];
}

// ---------------------------------------------------------------------------
// Section 4: a quaternion q = (q1, q2, q3, q4) with scalar part q4 is
// normalized by Algorithm 7 and turned into the rotation matrix of the unit
// quaternion.  The printed unit-norm matrix has two typos (2 q3^2 and 2 q2^2
// inside the first and last diagonal entries); the entries used here are the
// ones the general formula gives for |q| = 1:
//   R00 = 1 - 2 (q2^2 + q3^2)    R01 = 2 (q1 q2 - q3 q4)    R02 = 2 (q1 q3 + q2 q4)
//   R10 = 2 (q1 q2 + q3 q4)      R11 = 1 - 2 (q1^2 + q3^2)  R12 = 2 (q2 q3 - q1 q4)
//   R20 = 2 (q1 q3 - q2 q4)      R21 = 2 (q2 q3 + q1 q4)    R22 = 1 - 2 (q1^2 + q2^2)
// each evaluated as written, one rounded operation at a time.  R is stored
// row-major, 9 values per quaternion.  The zero quaternion gives
// q^ = (0, 0, 1, 0), the half turn about the third axis.
template <typename T>
__global__ void __launch_bounds__(256) k_rotation(const T* __restrict__ q, T* __restrict__ R, T* norm,
                                                   int64_t count) {
  using F = FP<T>;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
    T x[4], u[4], r, h;
#pragma unroll
    for (int k = 0; k < 4; ++k) x[k] = q[i * 4 + k];
    normalize_small<T, 4>(x, u, r, h, true);
    if (norm) norm[i] = r;
    const T q1 = u[0], q2 = u[1], q3 = u[2], q4 = u[3];
    const T two = T(2), one = T(1);
    const T q11 = F::mul(q1, q1), q22 = F::mul(q2, q2), q33 = F::mul(q3, q3);
    const T q12 = F::mul(q1, q2), q13 = F::mul(q1, q3), q23 = F::mul(q2, q3);
    const T q14 = F::mul(q1, q4), q24 = F::mul(q2, q4), q34 = F::mul(q3, q4);
    T* o = R + i * 9;
    o[0] = F::sub(one, F::mul(two, F::add(q22, q33)));
    o[1] = F::mul(two, F::sub(q12, q34));
    o[2] = F::mul(two, F::add(q13, q24));
    o[3] = F::mul(two, F::add(q12, q34));
    o[4] = F::sub(one, F::mul(two, F::add(q11, q33)));
    o[5] = F::mul(two, F::sub(q23, q14));
    o[6] = F::mul(two, F::sub(q13, q24));
    o[7] = F::mul(two, F::add(q23, q14));
    o[8] = F::sub(one, F::mul(two, F::add(q11, q22)));
  }
}

template <typename T>
cudaError_t launch_rotation(const T* q, T* R, T* norm, int64_t count, cudaStream_t s) {
  // a grid that covers the batch (one quaternion per thread), as the dense normalization kernels
  int64_t need = (count + 255) / 256;
  need = need < 1 ? 1 : (need < 2147483647 ? need : 2147483647);
  k_rotation<T><<<(int)need, 256, 0, s>>>(q, R, norm, count);
  return cudaGetLastError();
}
template cudaError_t launch_rotation<float>(const float*, float*, float*, int64_t, cudaStream_t);
template cudaError_t launch_rotation<double>(const double*, double*, double*, int64_t, cudaStream_t);

// ---------------------------------------------------------------------------
// Measurement aid: a streaming copy with 16-byte loads and stores, the
// achievable bandwidth ceiling for the same bytes.
// Warp tiles of 32 U consecutive 16-byte words over a covering grid, the
// layout of the quaternion kernel (k_small_vec16), so that the ceiling is
// taken with the same access pattern.
constexpr int COPY16_IN_FLIGHT = 6;
__global__ void __launch_bounds__(256) k_copy16(const uint4* __restrict__ src, uint4* __restrict__ dst, int64_t n16) {
  constexpr int U = COPY16_IN_FLIGHT;
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t w0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32 * U; w0 < n16; w0 += nw * 32 * U) {
    uint4 v[U];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (w0 + 32 * u + lane < n16) v[u] = __ldcs(src + w0 + 32 * u + lane);
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (w0 + 32 * u + lane < n16) __stcs(dst + w0 + 32 * u + lane, v[u]);
  }
}

__global__ void k_copy1(const unsigned char* __restrict__ src, unsigned char* __restrict__ dst, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) dst[i] = src[i];
}

cudaError_t launch_copy(void* dst, const void* src, int64_t bytes, cudaStream_t s) {
  const bool al = ((reinterpret_cast<uintptr_t>(dst) | reinterpret_cast<uintptr_t>(src)) & 15u) == 0 &&
                  (bytes % 16) == 0;
  if (al) {
    const int64_t n16 = bytes / 16;
    int64_t need = (n16 + 256 * COPY16_IN_FLIGHT - 1) / (256 * COPY16_IN_FLIGHT);
    need = need < 1 ? 1 : (need < 2147483647 ? need : 2147483647);
    k_copy16<<<(int)need, 256, 0, s>>>(reinterpret_cast<const uint4*>(src), reinterpret_cast<uint4*>(dst), n16);
  } else {
    k_copy1<<<device_sm_count() * 8, 256, 0, s>>>(reinterpret_cast<const unsigned char*>(src),
                                                  reinterpret_cast<unsigned char*>(dst), bytes);
  }
  return cudaGetLastError();
}

// The naive kernel's layout is that of the scaling kernels it is compared
// with (warp tiles of 32 U vectors, a covering grid, 6 vectors in flight).
constexpr int NAIVE_IN_FLIGHT = 6;

// Measurement aid: the naive algorithm the paper compares with in Table 4,
// y = x * (1 / sqrt(x1^2 + ... + xd^2)) with no scaling (it overflows and
// underflows where the scaling algorithms do not), for d <= 4.
template <typename T, int D>
__global__ void __launch_bounds__(256) k_naive(const T* __restrict__ x, T* __restrict__ y, int64_t count, int vec) {
  using F = FP<T>;
  constexpr int U = NAIVE_IN_FLIGHT;
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t w0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32 * U; w0 < count; w0 += nw * 32 * U) {
    T v[U][D];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = w0 + 32 * u + lane;
      if (i < count) {
        if constexpr (D * sizeof(T) == 16) {
          if (vec) { Vec<T, D>::load(x + i * D, v[u]); continue; }
        }
#pragma unroll
        for (int k = 0; k < D; ++k) v[u][k] = x[i * D + k];
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = w0 + 32 * u + lane;
      if (i < count) {
        T s = F::mul(v[u][0], v[u][0]);
#pragma unroll
        for (int k = 1; k < D; ++k) s = F::add(s, F::mul(v[u][k], v[u][k]));
        const T h = F::rcp(F::sqrt(s));
        T o[D];
#pragma unroll
        for (int k = 0; k < D; ++k) o[k] = F::mul(h, v[u][k]);
        if constexpr (D * sizeof(T) == 16) {
          if (vec) { Vec<T, D>::store(y + i * D, o); continue; }
        }
#pragma unroll
        for (int k = 0; k < D; ++k) y[i * D + k] = o[k];
      }
    }
  }
}

template <typename T, int D>
static cudaError_t launch_naive_d(const T* x, T* y, int64_t count, cudaStream_t s) {
  const int vec = (((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & 15u) == 0) ? 1 : 0;
  int64_t need = (count + 256 * NAIVE_IN_FLIGHT - 1) / (256 * NAIVE_IN_FLIGHT);
  need = need < 1 ? 1 : (need < 2147483647 ? need : 2147483647);
  k_naive<T, D><<<(int)need, 256, 0, s>>>(x, y, count, vec);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_naive(const T* x, T* y, int64_t count, int dim, cudaStream_t s) {
  switch (dim) {
    case 2: return launch_naive_d<T, 2>(x, y, count, s);
    case 3: return launch_naive_d<T, 3>(x, y, count, s);
    case 4: return launch_naive_d<T, 4>(x, y, count, s);
    default: return cudaErrorInvalidValue;
  }
}
template cudaError_t launch_naive<float>(const float*, float*, int64_t, int, cudaStream_t);
template cudaError_t launch_naive<double>(const double*, double*, int64_t, int, cudaStream_t);

// Binary64 multiply-add throughput probe: every thread runs FP64_PROBE_CHAINS
// independent chains a <- RN(RN(a * b) + c), `iters` steps each (two FP64
// instructions per step), and writes its results so nothing is removed.
constexpr int FP64_PROBE_CHAINS = 4;
constexpr int FP64_PROBE_THREADS = 256;

__global__ void __launch_bounds__(FP64_PROBE_THREADS) k_fp64_probe(double* out, int iters) {
  double a[FP64_PROBE_CHAINS];
  const double b = 1.0 + 0x1p-30 * (threadIdx.x & 7), c = 0x1p-40;
#pragma unroll
  for (int j = 0; j < FP64_PROBE_CHAINS; ++j) a[j] = 1.0 + j * 0x1p-20;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < FP64_PROBE_CHAINS; ++j) a[j] = __dadd_rn(__dmul_rn(a[j], b), c);
  }
  double r = 0.0;
#pragma unroll
  for (int j = 0; j < FP64_PROBE_CHAINS; ++j) r = __dadd_rn(r, a[j]);
  out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = r;
}

cudaError_t launch_fp64_probe(double* out, int blocks, int iters, cudaStream_t s) {
  k_fp64_probe<<<blocks, FP64_PROBE_THREADS, 0, s>>>(out, iters);
  return cudaGetLastError();
}

// Quotient algorithms on [count][3]: a tile of 256 vectors staged through
// shared memory (coalesced loads and stores of the AoS triples), one vector
// per thread.
template <typename T, int ALG>
__global__ void __launch_bounds__(256) k_quotient3(const T* __restrict__ x, T* y, T* norm, int64_t count) {
  constexpr int NT = 256;
  __shared__ T tile[NT * 3];
  const int t = threadIdx.x;
  for (int64_t v0 = (int64_t)blockIdx.x * NT; v0 < count; v0 += (int64_t)gridDim.x * NT) {
    const int nv = (int)((count - v0) < NT ? (count - v0) : NT);
    const T* src = x + v0 * 3;
    for (int i = t; i < nv * 3; i += NT) tile[i] = __ldcs(src + i);
    __syncthreads();
    T yv[3], r = T(0);
    if (t < nv) {
      const T xv[3] = {tile[3 * t], tile[3 * t + 1], tile[3 * t + 2]};
      if (ALG == 1) quotient1_3<T>(xv, yv, r);
      else quotient2_3<T>(xv, yv, r);
      if (norm) norm[v0 + t] = r;
    }
    __syncthreads();
    if (t < nv) {
      tile[3 * t] = yv[0];
      tile[3 * t + 1] = yv[1];
      tile[3 * t + 2] = yv[2];
    }
    __syncthreads();
    T* dst = y + v0 * 3;
    for (int i = t; i < nv * 3; i += NT) __stcs(dst + i, tile[i]);
    __syncthreads();
  }
}

template <typename T>
cudaError_t launch_quotient3(const T* x, T* y, T* norm, int64_t count, int alg, cudaStream_t s) {
  // a grid that covers the batch (one tile of 256 vectors per block), the launch shape of the
  // scaling kernels it is compared with (Table 3)
  int64_t need = (count + 255) / 256;
  need = need < 1 ? 1 : (need < 2147483647 ? need : 2147483647);
  const int grid = (int)need;
  if (alg == 1) k_quotient3<T, 1><<<grid, 256, 0, s>>>(x, y, norm, count);
  else k_quotient3<T, 2><<<grid, 256, 0, s>>>(x, y, norm, count);
  return cudaGetLastError();
}
template cudaError_t launch_quotient3<float>(const float*, float*, float*, int64_t, int, cudaStream_t);
template cudaError_t launch_quotient3<double>(const double*, double*, double*, int64_t, int, cudaStream_t);

}  // namespace ngb
