// ngb_threadpath.cuh -- a short vector (n <= 16) by one thread: the ragged
// thread items, forward (Algorithms 5-7 for n <= 4, the generic steps in the
// order CR(n) otherwise) and backward (dot = y . g, left to right for n <= 4,
// the order CR(n) otherwise; grad_k = ((g_k - y_k dot) h) c).
#pragma once
#include "ngb_rowpath.cuh"

namespace ngb {

// binary64 thread items with their products on the integer pipes
// (thread_item_bwd_f64).  Ragged binary64 forward + backward per step:
// 1.513-1.523 ms against 1.536-1.538 ms with the hardware products.
constexpr bool THREAD_BWD_F64_INT = true;

// One vector of n <= 16 components by one thread (vector zero rule for n = 4).
template <typename T>
__device__ __forceinline__ void thread_item_fwd(const T* __restrict__ xr, T* yr, int n, const VecOut<T>& out,
                                                int64_t vec) {
  T r, h;
  int code;
  if (n <= 4) {
    T xv[4], yv[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) xv[k] = k < n ? xr[k] : T(0);
    bool done = false;
    if constexpr (sizeof(T) == 8 && SMALL_F64_INTEGER) {  // one integer-pipe form for every n <= 4
      const SmallKeysF64<4> kk(xv);
      if (kk.ok) {
        code = normalize_small_f64_int<4>(xv, yv, r, h, false, kk);
        done = true;
      }
    }
    if (!done) {
      switch (n) {
        case 1: code = normalize_small_hw<T, 1>(xv, yv, r, h, false); break;
        case 2: code = normalize_small_hw<T, 2>(xv, yv, r, h, false); break;
        case 3: code = normalize_small_hw<T, 3>(xv, yv, r, h, false); break;
        default: code = normalize_small_hw<T, 4>(xv, yv, r, h, false); break;
      }
    }
    if (yr) {
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (k < n) yr[k] = yv[k];
    }
  } else {
    code = normalize_thread_generic<T, 16>(xr, yr, n, r, h);
  }
  out.put(vec, r, h, code);
}

// Backward of one thread item with the hardware operations (every product
// and sum on the FP64 pipe).
template <typename T>
__device__ __forceinline__ void thread_item_bwd_hw(const T* __restrict__ yr, const T* __restrict__ gr, T* gradr,
                                                   int n, T h, int code) {
  if (n <= 4) {
    T yv[4], gv[4], o[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      yv[k] = k < n ? yr[k] : T(0);
      gv[k] = k < n ? gr[k] : T(0);
    }
    switch (n) {
      case 1: backward_small<T, 1>(yv, gv, h, code, o); break;
      case 2: backward_small<T, 2>(yv, gv, h, code, o); break;
      case 3: backward_small<T, 3>(yv, gv, h, code, o); break;
      default: backward_small<T, 4>(yv, gv, h, code, o); break;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (k < n) gradr[k] = o[k];
  } else {
    backward_thread_generic<T, 16>(yr, gr, n, h, code, gradr);
  }
}

template <typename T>
__device__ __noinline__ void thread_item_bwd_hw_call(const T* __restrict__ yr, const T* __restrict__ gr, T* gradr,
                                                     int n, T h, int code) {
  thread_item_bwd_hw<T>(yr, gr, gradr, n, h, code);
}

// The same for binary64 with every product on the integer pipes: y_k g_k
// and y_k dot by f64emu::mul_signed and, with c = 1, d_k h by f64emu::mul,
// when the vector's integer keys put them in range (products_in_range,
// grad_h_in_range, as in the warp and group backward); the sums stay on the
// FP64 pipe.  Any other vector takes the hardware form, out of line.  The
// thread backward kernel leaves the ALU almost idle and the FP64 pipe busy,
// so all three products move to the integer pipes.  Same bits in every case.
__device__ __forceinline__ void thread_item_bwd_f64(const double* __restrict__ yr, const double* __restrict__ gr,
                                                    double* gradr, int n, double h, int code) {
  constexpr int NMAX = 16;
  if (code == CODE_ZERO) {
    for (int k = 0; k < n; ++k) gradr[k] = 0.0;
    return;
  }
  auto bits = [](double v) { return static_cast<uint64_t>(__double_as_longlong(v)); };
  auto dbl = [](uint64_t b) { return __longlong_as_double(static_cast<long long>(b)); };
  double q[NMAX];
  MagTrack<double> ry, rg;
#pragma unroll
  for (int k = 0; k < NMAX; ++k) {
    const double yk = k < n ? yr[k] : 0.0, gk = k < n ? gr[k] : 0.0;  // zero padding changes no key
    ry.take(yk);
    rg.take(gk);
    q[k] = dbl(f64emu::mul_signed(bits(yk), bits(gk)));  // used only when in range (checked next)
  }
  if (code != CODE_ONE || !products_in_range(ry, rg)) {
    thread_item_bwd_hw_call<double>(yr, gr, gradr, n, h, code);
    return;
  }
  double dot;
  if (n <= 4) {  // left to right (Algorithms 3-7's order for the sum of squares)
    dot = q[0];
#pragma unroll
    for (int k = 1; k < 4; ++k)
      if (k < n) dot = FP<double>::add(dot, q[k]);
  } else {
    dot = cr_sum_thread<double, NMAX>(q, n);
  }
  MagTrack<double> rd;
  rd.take(dot);
  if (!products_in_range(ry, rd)) {
    thread_item_bwd_hw_call<double>(yr, gr, gradr, n, h, code);
    return;
  }
  const uint64_t db = bits(dot), hb = bits(h);
  if (grad_h_in_range(ry, rg, rd, h)) {
#pragma unroll
    for (int k = 0; k < NMAX; ++k)
      if (k < n) {
        const double d = FP<double>::sub(gr[k], dbl(f64emu::mul_signed(bits(yr[k]), db)));
        gradr[k] = dbl(f64emu::mul(bits(d), hb));
      }
  } else {
#pragma unroll
    for (int k = 0; k < NMAX; ++k)
      if (k < n) gradr[k] = FP<double>::mul(FP<double>::sub(gr[k], dbl(f64emu::mul_signed(bits(yr[k]), db))), h);
  }
}

template <typename T>
__device__ __forceinline__ void thread_item_bwd(const T* __restrict__ yr, const T* __restrict__ gr, T* gradr, int n,
                                                T h, int code) {
  if constexpr (sizeof(T) == 8 && THREAD_BWD_F64_INT) thread_item_bwd_f64(yr, gr, gradr, n, h, code);
  else thread_item_bwd_hw<T>(yr, gr, gradr, n, h, code);
}

}  // namespace ngb
