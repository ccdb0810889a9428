// kernels_fixed.cuh -- dense [count][dim] batches: forward and backward
// kernels and their launchers, instantiated per precision by fixed_f32.cu and
// fixed_f64.cu.
//
//   dim <= 4           one vector per thread (Algorithms 5-7); 16-byte vector
//                      loads when a vector is 16 bytes (binary32 quaternions,
//                      binary64 pairs) or two of them (binary64 quaternions),
//                      otherwise one load per component (a warp's loads cover
//                      consecutive lines; L1 serves the repeats).
//   5 <= dim <= 16     one vector per thread, order CR(n).
//   17 <= dim <= 128   one row per group of 8 or 16 lanes, held in registers
//                      (binary64: up to 64; 65..128 as the longer rows).
//   129 <= dim <= 1024 one warp per row held in registers, 16-byte loads when
//                      rows are 16-byte aligned (binary32: one row per
//                      half-warp for 129..256).
//   1024 < dim <= 16384  one warp per row streaming it (three passes).
//   dim > 16384        one block of 256 threads per row streaming it.
#pragma once
#include "ngb_internal.h"
#include "ngb_grouppath.cuh"

namespace ngb {

constexpr int SMALL_THREADS = 256;
// 16-byte vectors in flight per thread in k_small_vec16 and k_small_bwd.
// Measured on 2^26 binary32 quaternions (three interleaved repeats): 4 in
// flight 0.89 of the copy bandwidth, 5: 0.93, 6: 0.967, 7: 0.961, 8: 0.935;
// the backward (two 16-byte loads per quaternion) is best at 4 (6: 0.83).
constexpr int VEC16_IN_FLIGHT = 6;
constexpr int BWD16_IN_FLIGHT = 4;
// rows per warp with their loads in flight together in k_rows_warp (measured
// on 2^20 binary32 rows of 256: 1 row 0.887 of the copy bandwidth, 2: 0.861,
// 3: 0.874, 4: 0.855)
constexpr int ROWS_IN_FLIGHT = 1;
// binary32 rows of 129..256 on half-warps (k_rows_half)
constexpr bool ROWS_HALF_WARP = true;

// ---------------------------------------------------------------------------
// dim <= 4, one 16-byte vector per thread, U vectors in flight per thread.
// Layout: each warp takes a tile of 32 U consecutive vectors (lane l holds
// vectors l, 32 + l, ..., so that each of the U loads of a warp covers 512
// contiguous bytes), and the grid covers the whole batch (one tile per warp;
// the loop only matters when the grid is capped).  Measured on 2^26 binary32
// quaternions against the earlier layout (one full wave of persistent
// threads, thread t taking vectors t, t + S, ... for the grid size S): 0.996
// of the measured HBM copy bandwidth against 0.953; warp tiles with the
// persistent grid 0.94-0.95, the persistent layout with the covering grid
// 0.965; torch's device copy of the same bytes 0.999.  The tile loop is
// warp-uniform, so binary64 (normalize_small_warp) can vote per warp; lanes
// past the end load zeros and write nothing.
template <typename T, int D>
__global__ void __launch_bounds__(SMALL_THREADS) k_small_vec16(const T* __restrict__ x, T* y, VecOut<T> out,
                                                                int64_t count, int quat_zero) {
  static_assert(D * sizeof(T) == 16, "one 16-byte vector per element vector");
  constexpr int U = VEC16_IN_FLIGHT;
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t w0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32 * U; w0 < count;
       w0 += nw * 32 * U) {
    T xv[U][D];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = w0 + 32 * u + lane;
      if (i < count) {
        Vec<T, D>::load(x + i * D, xv[u]);
      } else {
#pragma unroll
        for (int k = 0; k < D; ++k) xv[u][k] = T(0);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = w0 + 32 * u + lane;
      if constexpr (sizeof(T) == 4) {
        if (i < count) {
          T yv[D], r, h;
          const int code = normalize_small<T, D>(xv[u], yv, r, h, quat_zero != 0);
          if (y) Vec<T, D>::store(y + i * D, yv);
          out.put(i, r, h, code);
        }
      } else if (w0 + 32 * u < count) {  // warp-uniform
        T yv[D], r, h;
        const int code = normalize_small_warp<T, D>(xv[u], yv, r, h, quat_zero != 0, i < count);
        if (i < count) {
          if (y) Vec<T, D>::store(y + i * D, yv);
          out.put(i, r, h, code);
        }
      }
    }
  }
}

// dim <= 4, one vector per thread read and written as D scalars (a warp's
// loads cover consecutive 128-byte lines; L1 serves the repeated lines), U
// vectors in flight per thread: for D = 1, 2, 3 and unaligned quaternions.
// binary64 takes one vector at a time: its integer-pipe steps are long, and
// fewer registers give more warps (measured on 2^25 quaternions: U = 4
// 1.34 ms, 2 1.18 ms, 1 1.18 ms, 8 1.55 ms; with the FP64 squares, U = 2
// 0.882 ms against 0.871 ms).  binary32 (2^24 three-component vectors, warp
// tiles): U = 2 0.088 ms, 4 0.0724 ms, 6 0.0716 ms, 8 0.080 ms.
template <typename T> constexpr int SMALL_DIRECT_IN_FLIGHT = sizeof(T) == 8 ? 1 : 6;
// pairs (binary64, D = 4, x and y 16-byte aligned): each quaternion is read
// and written as two 16-byte pairs instead of four scalars.  On device memory
// L1 serves the repeated lines of the scalar form either way; on pinned host
// memory (zero-copy) the scalar form fetched each line again over the host
// link and ran 2.2 times slower than staging the copies.
// Layout as k_small_vec16: warp tiles of 32 U consecutive vectors over a
// covering grid (the loop is warp-uniform; binary64 votes per warp).
template <typename T, int D>
__global__ void __launch_bounds__(SMALL_THREADS) k_small_direct(const T* __restrict__ x, T* y, VecOut<T> out,
                                                                 int64_t count, int quat_zero, int pairs) {
  constexpr int U = SMALL_DIRECT_IN_FLIGHT<T>;
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t w0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32 * U; w0 < count;
       w0 += nw * 32 * U) {
    T xv[U][D];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = w0 + 32 * u + lane;
      if constexpr (D == 4 && sizeof(T) == 8) {
        if (pairs) {  // uniform over the launch
          if (i < count) {
            Vec<T, 2>::load(x + i * D, xv[u]);
            Vec<T, 2>::load(x + i * D + 2, xv[u] + 2);
          } else {
#pragma unroll
            for (int k = 0; k < D; ++k) xv[u][k] = T(0);
          }
          continue;
        }
      }
#pragma unroll
      for (int k = 0; k < D; ++k) xv[u][k] = i < count ? __ldcs(x + i * D + k) : T(0);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = w0 + 32 * u + lane;
      if (w0 + 32 * u >= count) break;  // warp-uniform
      T yv[D], r, h;
      const int code = normalize_small_warp<T, D>(xv[u], yv, r, h, quat_zero != 0, i < count);
      if (i < count) {
        if (y) {
          if constexpr (D == 4 && sizeof(T) == 8) {
            if (pairs) {
              Vec<T, 2>::store(y + i * D, yv);
              Vec<T, 2>::store(y + i * D + 2, yv + 2);
              out.put(i, r, h, code);
              continue;
            }
          }
#pragma unroll
          for (int k = 0; k < D; ++k) __stcs(y + i * D + k, yv[k]);
        }
        out.put(i, r, h, code);
      }
    }
  }
}


template <typename T, int D>
__global__ void __launch_bounds__(SMALL_THREADS) k_small_bwd(const T* __restrict__ y, const T* __restrict__ g,
                                                              const T* __restrict__ hs, const int8_t* __restrict__ cs,
                                                              T* grad, int64_t count, int vec16) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  if constexpr (D * sizeof(T) == 16) {
    if (vec16) {  // BWD16_IN_FLIGHT vectors of y and g (16 bytes each) in flight per thread, warp tiles
      constexpr int U = BWD16_IN_FLIGHT;
      const int lane = threadIdx.x & 31;
      const int64_t nw = stride >> 5;
      for (int64_t w0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32 * U; w0 < count;
           w0 += nw * 32 * U) {
        T yv[U][D], gv[U][D], hv[U];
        int cv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int64_t i = w0 + 32 * u + lane;
          if (i < count) {
            Vec<T, D>::load(y + i * D, yv[u]);
            Vec<T, D>::load(g + i * D, gv[u]);
            hv[u] = hs[i];
            cv[u] = cs[i];
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int64_t i = w0 + 32 * u + lane;
          if (i < count) {
            T o[D];
            backward_small<T, D>(yv[u], gv[u], hv[u], cv[u], o);
            Vec<T, D>::store(grad + i * D, o);
          }
        }
      }
      return;
    }
  }
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
    T yv[D], gv[D], o[D];
#pragma unroll
    for (int k = 0; k < D; ++k) { yv[k] = y[i * D + k]; gv[k] = g[i * D + k]; }
    backward_small<T, D>(yv, gv, hs[i], cs[i], o);
#pragma unroll
    for (int k = 0; k < D; ++k) grad[i * D + k] = o[k];
  }
}

// ---------------------------------------------------------------------------
// 5 <= dim <= 16, one row per thread.
template <typename T>
__global__ void __launch_bounds__(256) k_rows_thread(const T* __restrict__ x, T* y, VecOut<T> out, int64_t count,
                                                      int n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
    T r, h;
    const int code = normalize_thread_generic<T, 16>(x + i * n, y ? y + i * n : nullptr, n, r, h);
    out.put(i, r, h, code);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_rows_thread_bwd(const T* __restrict__ y, const T* __restrict__ g,
                                                          const T* __restrict__ hs, const int8_t* __restrict__ cs,
                                                          T* grad, int64_t count, int n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride)
    backward_thread_generic<T, 16>(y + i * n, g + i * n, n, hs[i], cs[i], grad + i * n);
}

// 17 <= dim <= 1024, one warp per row (grid-stride over rows).
template <typename T, int V, int CH>
__global__ void __launch_bounds__(256) k_rows_warp(const T* __restrict__ x, T* y, VecOut<T> out, int64_t count,
                                                    int n) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  // ROWS_IN_FLIGHT rows per warp: their loads are all issued before the first
  // row is reduced
  constexpr int R = ROWS_IN_FLIGHT;
  for (int64_t row0 = w0; row0 < count; row0 += nw * R) {
    T v[R][CH][V];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int64_t row = row0 + r * nw;
      if (row < count) warp_load<T, V, CH>(x + row * n, n, lane, v[r]);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int64_t row = row0 + r * nw;
      if (row < count) warp_forward_loaded<T, V, CH>(v[r], x + row * n, y ? y + row * n : nullptr, n, lane, out, row);
    }
  }
}

// 17 <= dim <= 8 W: one row per group of W = 8 or 16 lanes (group_forward,
// csrc/ngb_grouppath.cuh), 32 / W rows per warp, the rows held in registers.
// One warp per row of this length leaves most lanes idle in the per-row
// steps (tree levels, square root, reciprocal) and in the loads of a short
// row.
template <typename T, int W>
__global__ void __launch_bounds__(256) k_rows_group(const T* __restrict__ x, T* y, VecOut<T> out, int64_t count,
                                                     int n) {
  constexpr int PER = 32 / W;
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r0 = w0 * PER; r0 < count; r0 += nw * PER) {
    const int64_t row = r0 + lane / W;
    if (row < count) group_forward<T, W>(x + row * n, y ? y + row * n : nullptr, n, lane, out, row);
  }
}

template <typename T, int W>
__global__ void __launch_bounds__(256) k_rows_group_bwd(const T* __restrict__ y, const T* __restrict__ g,
                                                         const T* __restrict__ hs, const int8_t* __restrict__ cs,
                                                         T* grad, int64_t count, int n) {
  constexpr int PER = 32 / W;
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r0 = w0 * PER; r0 < count; r0 += nw * PER) {
    const int64_t row = r0 + lane / W;
    if (row < count) group_backward<T, W>(y + row * n, g + row * n, grad + row * n, n, lane, hs[row], cs[row]);
  }
}

// binary32 rows of 128 < dim <= 256 (multiple of 4, 16-byte aligned): one
// row per half-warp (half_forward_f32), two rows per warp.
template <int CH>
__global__ void __launch_bounds__(256) k_rows_half(const float* __restrict__ x, float* y, VecOut<float> out,
                                                   int64_t count, int n) {
  const int lane = threadIdx.x & 31, half = lane >> 4, hl = lane & 15;
  const unsigned gmask = half ? 0xFFFF0000u : 0x0000FFFFu;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r0 = 2 * w0; r0 < count; r0 += 2 * nw) {
    const int64_t row = r0 + half;
    const bool valid = row < count;
    const int64_t rr = valid ? row : r0;  // the second half of a last, odd pair repeats row r0 without output
    half_forward_f32<CH>(x + rr * n, (valid && y) ? y + rr * n : nullptr, n, hl, gmask, out, rr, valid);
  }
}

template <typename T, int V, int CH>
__global__ void __launch_bounds__(256) k_rows_warp_bwd(const T* __restrict__ y, const T* __restrict__ g,
                                                        const T* __restrict__ hs, const int8_t* __restrict__ cs,
                                                        T* grad, int64_t count, int n) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t row = w0; row < count; row += nw)
    warp_backward<T, V, CH>(y + row * n, g + row * n, grad + row * n, n, lane, hs[row], cs[row]);
}

// 1024 < dim <= 16384, one warp per row streaming it.
// binary64 rows of 17 <= dim <= 16384: one warp streams NB consecutive rows
// and shares one square root and reciprocal among them.
constexpr int F64_ROW_BATCH = 4;

// The dense binary64 row batch forms 3 of every 8 outputs on the integer
// pipe (see F64_EMU_OUTPUTS_OF_8).
constexpr int F64_EMU_OUTPUTS_OF_8_ROWS = 3;

template <typename T, int NB>
__global__ void __launch_bounds__(256) k_rows_stream_batch(const T* __restrict__ x, T* y, VecOut<T> out,
                                                            int64_t count, int n) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t g = w0 * NB; g < count; g += nw * NB) {
    const int nb = (int)((count - g) < NB ? (count - g) : NB);
    auto item = [&](int j, const T*& xr, T*& yr, int& nn, int64_t& vec) {
      vec = g + j;
      xr = x + vec * n;
      yr = y ? y + vec * n : nullptr;
      nn = n;
    };
    warp_forward_stream_batch<T, NB, MAX_LEN, false, F64_EMU_OUTPUTS_OF_8_ROWS>(item, nb, lane, out);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_rows_stream(const T* __restrict__ x, T* y, VecOut<T> out, int64_t count,
                                                      int n) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t row = w0; row < count; row += nw)
    warp_forward_stream<T>(x + row * n, y ? y + row * n : nullptr, n, lane, out, row);
}

template <typename T>
__global__ void __launch_bounds__(256) k_rows_stream_bwd(const T* __restrict__ y, const T* __restrict__ g,
                                                          const T* __restrict__ hs, const int8_t* __restrict__ cs,
                                                          T* grad, int64_t count, int n) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t row = w0; row < count; row += nw)
    warp_backward_stream<T>(y + row * n, g + row * n, grad + row * n, n, lane, hs[row], cs[row]);
}

// dim > 16384, one block of 256 threads per row streaming it.
template <typename T>
__global__ void __launch_bounds__(256) k_rows_block(const T* __restrict__ x, T* y, VecOut<T> out, int64_t count,
                                                     int n) {
  __shared__ BlockShared<T, 256> sh;
  for (int64_t row = blockIdx.x; row < count; row += gridDim.x)
    block_forward_stream<T, 256>(x + row * n, y ? y + row * n : nullptr, n, out, row, sh);
}

template <typename T>
__global__ void __launch_bounds__(256) k_rows_block_bwd(const T* __restrict__ y, const T* __restrict__ g,
                                                         const T* __restrict__ hs, const int8_t* __restrict__ cs,
                                                         T* grad, int64_t count, int n) {
  __shared__ BlockShared<T, 256> sh;
  for (int64_t row = blockIdx.x; row < count; row += gridDim.x)
    block_backward_stream<T, 256>(y + row * n, g + row * n, grad + row * n, n, hs[row], cs[row], sh);
}

// ---------------------------------------------------------------------------
// Launchers
inline bool aligned16(const void* p) { return p == nullptr || (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Blocks that cover work_items at items_per_block each (at most 2^31 - 1).
inline int grid_cover(int64_t work_items, int64_t items_per_block) {
  int64_t need = (work_items + items_per_block - 1) / items_per_block;
  if (need < 1) need = 1;
  return (int)(need < 2147483647 ? need : 2147483647);
}

template <typename K>
inline int grid_for(K kernel, int threads, int64_t work_items, int items_per_block) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0);
  if (per_sm < 1) per_sm = 1;
  int64_t need = (work_items + items_per_block - 1) / items_per_block;
  int64_t cap = (int64_t)device_sm_count() * per_sm;
  if (need < 1) need = 1;
  return (int)(need < cap ? need : cap);
}

template <typename T, int D>
cudaError_t launch_small_fwd(const T* x, T* y, VecOut<T> out, int64_t count, bool quat_zero, cudaStream_t s) {
  const bool vec16 = aligned16(x) && aligned16(y);
  if constexpr (sizeof(T) == 4 && D == 4) {  // opt-in: quat_bulk_enabled()
    if (count > 0 && quat_bulk_enabled()) {
      const cudaError_t e = launch_quat_bulk(x, y, out, count, quat_zero, s);
      if (e != cudaErrorNotSupported) return e;
    }
  }
  if constexpr (D * sizeof(T) == 16) {
    if (vec16) {
      auto k = k_small_vec16<T, D>;
      k<<<grid_cover(count, SMALL_THREADS * VEC16_IN_FLIGHT), SMALL_THREADS, 0, s>>>(x, y, out, count, quat_zero);
      return cudaGetLastError();
    }
  }
  {
    auto k = k_small_direct<T, D>;
    const int pairs = (sizeof(T) == 8 && D == 4 && vec16) ? 1 : 0;
    k<<<grid_cover(count, SMALL_THREADS * SMALL_DIRECT_IN_FLIGHT<T>), SMALL_THREADS, 0, s>>>(x, y, out, count,
                                                                                            quat_zero, pairs);
  }
  return cudaGetLastError();
}

template <typename T, int D>
cudaError_t launch_small_bwd(const T* y, const T* g, const T* h, const int8_t* c, T* grad, int64_t count,
                             cudaStream_t s) {
  const bool vec16 = aligned16(y) && aligned16(g) && aligned16(grad);
  auto k = k_small_bwd<T, D>;
  // the 16-byte path takes warp tiles of 32 BWD16_IN_FLIGHT vectors over a covering grid
  const int grid = (D * sizeof(T) == 16 && vec16) ? grid_cover(count, SMALL_THREADS * BWD16_IN_FLIGHT)
                                                  : grid_for(k, SMALL_THREADS, count, SMALL_THREADS * 4);
  k<<<grid, SMALL_THREADS, 0, s>>>(y, g, h, c, grad, count, vec16 ? 1 : 0);
  return cudaGetLastError();
}

// Number of 32*V-element chunks per lane: the smallest power of two covering n.
inline int chunks_for(int n, int per_chunk) {
  int ch = 1;
  while (ch * per_chunk < n) ch *= 2;
  return ch;
}

template <typename T, int V, int CH>
cudaError_t launch_warp_rows(const T* x, T* y, VecOut<T> out, int64_t count, int n, cudaStream_t s) {
  auto k = k_rows_warp<T, V, CH>;
  // rows of several chunks per lane: a covering grid (binary32 rows of 1000: 0.344 -> 0.304 ms per
  // GiB); shorter rows keep one persistent wave
  const int grid = CH >= 4 ? grid_cover(count, 8) : grid_for(k, 256, count, 8);
  k<<<grid, 256, 0, s>>>(x, y, out, count, n);
  return cudaGetLastError();
}

template <typename T, int V, int CH>
cudaError_t launch_warp_rows_bwd(const T* y, const T* g, const T* h, const int8_t* c, T* grad, int64_t count, int n,
                                 cudaStream_t s) {
  auto k = k_rows_warp_bwd<T, V, CH>;
  const int grid = grid_for(k, 256, count, 8);
  k<<<grid, 256, 0, s>>>(y, g, h, c, grad, count, n);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fixed_forward_impl(const T* x, T* y, VecOut<T> out, int64_t count, int dim, bool quat_zero,
                                      cudaStream_t s) {
  constexpr int W = 16 / sizeof(T);  // binary32 register rows: 16-byte loads when aligned
  switch (dim) {
    case 1: return launch_small_fwd<T, 1>(x, y, out, count, false, s);
    case 2: return launch_small_fwd<T, 2>(x, y, out, count, false, s);
    case 3: return launch_small_fwd<T, 3>(x, y, out, count, false, s);
    case 4: return launch_small_fwd<T, 4>(x, y, out, count, quat_zero, s);
    default: break;
  }
  if (dim <= 16) {
    auto k = k_rows_thread<T>;
    k<<<grid_cover(count, 256), 256, 0, s>>>(x, y, out, count, dim);
    return cudaGetLastError();
  }
  // groups of 8 (dim <= 64) or 16 lanes, one row each, a covering grid; binary64 rows of 65..128
  // keep the 4-row streaming batch, which shares one square root and reciprocal among 4 rows
  // (measured per GiB of rows: binary32 dim 40 1.70 -> 0.62 ms, dim 100 0.74 -> 0.52 ms; binary64
  // dim 17 9.22 -> 4.03 ms, dim 100 1.72 ms on the batch against 1.89 ms on groups of 16)
  if (dim <= (sizeof(T) == 4 ? 128 : 64)) {
    if (dim <= 64) k_rows_group<T, 8><<<grid_cover(count, 32), 256, 0, s>>>(x, y, out, count, dim);
    else k_rows_group<T, 16><<<grid_cover(count, 16), 256, 0, s>>>(x, y, out, count, dim);
    return cudaGetLastError();
  }
  if constexpr (sizeof(T) == 8) {  // binary64: streaming warps, 4 rows per warp (integer-pipe steps)
    if (dim <= 16384) {
      auto k = k_rows_stream_batch<T, F64_ROW_BATCH>;
      k<<<grid_cover((count + F64_ROW_BATCH - 1) / F64_ROW_BATCH, 8), 256, 0, s>>>(x, y, out, count, dim);
      return cudaGetLastError();
    }
  } else {
    if (ROWS_HALF_WARP && dim > 128 && dim <= 256 && dim % 4 == 0 && aligned16(x) && (!y || aligned16(y))) {
      // a covering grid (one row pair per warp), not one persistent wave: measured on 2^20 rows of
      // 256, 1.04 against 0.90 of the measured HBM copy bandwidth
      auto k = k_rows_half<4>;
      k<<<grid_cover((count + 1) / 2, 8), 256, 0, s>>>(x, y, out, count, dim);
      return cudaGetLastError();
    }
    if (dim <= 1024) {
    if (W > 1 && (dim % W == 0) && aligned16(x) && aligned16(y)) {
      switch (chunks_for(dim, 32 * W)) {
        case 1: return launch_warp_rows<T, W, 1>(x, y, out, count, dim, s);
        case 2: return launch_warp_rows<T, W, 2>(x, y, out, count, dim, s);
        case 4: return launch_warp_rows<T, W, 4>(x, y, out, count, dim, s);
        case 8: return launch_warp_rows<T, W, 8>(x, y, out, count, dim, s);
        default: return launch_warp_rows<T, W, 32 / W>(x, y, out, count, dim, s);
      }
    }
    switch (chunks_for(dim, 32)) {
      case 1: return launch_warp_rows<T, 1, 1>(x, y, out, count, dim, s);
      case 2: return launch_warp_rows<T, 1, 2>(x, y, out, count, dim, s);
      case 4: return launch_warp_rows<T, 1, 4>(x, y, out, count, dim, s);
      case 8: return launch_warp_rows<T, 1, 8>(x, y, out, count, dim, s);
      case 16: return launch_warp_rows<T, 1, 16>(x, y, out, count, dim, s);
      default: return launch_warp_rows<T, 1, 32>(x, y, out, count, dim, s);
    }
    }
    if (dim <= 16384) {
      auto k = k_rows_stream<T>;
      k<<<grid_cover(count, 8), 256, 0, s>>>(x, y, out, count, dim);
      return cudaGetLastError();
    }
  }
  auto k = k_rows_block<T>;
  k<<<grid_for(k, 256, count, 1), 256, 0, s>>>(x, y, out, count, dim);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fixed_backward_impl(const T* y, const T* g, const T* h, const int8_t* c, T* grad, int64_t count,
                                       int dim, cudaStream_t s) {
  // binary32 rows use 16-byte loads; binary64 rows use 8-byte loads, whose
  // slot layout needs fewer additions in the summation tree (5 shuffle levels
  // and 7 in-lane additions instead of 5 x 2 and 7)
  constexpr int W = sizeof(T) == 4 ? 4 : 1;
  switch (dim) {
    case 1: return launch_small_bwd<T, 1>(y, g, h, c, grad, count, s);
    case 2: return launch_small_bwd<T, 2>(y, g, h, c, grad, count, s);
    case 3: return launch_small_bwd<T, 3>(y, g, h, c, grad, count, s);
    case 4: return launch_small_bwd<T, 4>(y, g, h, c, grad, count, s);
    default: break;
  }
  if (dim <= 16) {
    auto k = k_rows_thread_bwd<T>;
    k<<<grid_for(k, 256, count, 256), 256, 0, s>>>(y, g, h, c, grad, count, dim);
    return cudaGetLastError();
  }
  if (dim <= (sizeof(T) == 4 ? 128 : 64)) {  // as the forward: groups of 8 or 16 lanes
    if (dim <= 64) k_rows_group_bwd<T, 8><<<grid_cover(count, 32), 256, 0, s>>>(y, g, h, c, grad, count, dim);
    else k_rows_group_bwd<T, 16><<<grid_cover(count, 16), 256, 0, s>>>(y, g, h, c, grad, count, dim);
    return cudaGetLastError();
  }
  if (dim <= 1024) {
    if (W > 1 && (dim % W == 0) && aligned16(y) && aligned16(g) && aligned16(grad)) {
      switch (chunks_for(dim, 32 * W)) {
        case 1: return launch_warp_rows_bwd<T, W, 1>(y, g, h, c, grad, count, dim, s);
        case 2: return launch_warp_rows_bwd<T, W, 2>(y, g, h, c, grad, count, dim, s);
        case 4: return launch_warp_rows_bwd<T, W, 4>(y, g, h, c, grad, count, dim, s);
        case 8: return launch_warp_rows_bwd<T, W, 8>(y, g, h, c, grad, count, dim, s);
        default: return launch_warp_rows_bwd<T, W, 32 / W>(y, g, h, c, grad, count, dim, s);
      }
    }
    switch (chunks_for(dim, 32)) {
      case 1: return launch_warp_rows_bwd<T, 1, 1>(y, g, h, c, grad, count, dim, s);
      case 2: return launch_warp_rows_bwd<T, 1, 2>(y, g, h, c, grad, count, dim, s);
      case 4: return launch_warp_rows_bwd<T, 1, 4>(y, g, h, c, grad, count, dim, s);
      case 8: return launch_warp_rows_bwd<T, 1, 8>(y, g, h, c, grad, count, dim, s);
      case 16: return launch_warp_rows_bwd<T, 1, 16>(y, g, h, c, grad, count, dim, s);
      default: return launch_warp_rows_bwd<T, 1, 32>(y, g, h, c, grad, count, dim, s);
    }
  }
  if (dim <= 16384) {
    auto k = k_rows_stream_bwd<T>;
    k<<<grid_for(k, 256, count, 8), 256, 0, s>>>(y, g, h, c, grad, count, dim);
  } else {
    auto k = k_rows_block_bwd<T>;
    k<<<grid_for(k, 256, count, 1), 256, 0, s>>>(y, g, h, c, grad, count, dim);
  }
  return cudaGetLastError();
}

}  // namespace ngb
