// ngb_grouppath.cuh -- short vectors by groups of W = 8 or 16 lanes, 32 / W
// vectors per warp, each vector held in registers (n <= 8 W).
//
// On GB300 a binary64 instruction costs the FP64 pipe about the same whether
// one lane or 32 lanes execute it.  A warp that normalizes one short vector
// spends most of its per-vector steps -- the square root and reciprocal of
// the sum, the shuffle levels of the summation tree, the backward's tree --
// on lanes that have nothing to do.  A group of W lanes per vector lets one
// warp instruction serve 32 / W vectors in those steps.
//
// Layout: lane g (0 <= g < W) of a group holds the terms k = W c + g,
// c = 0 .. 7, in q[c].  With n <= 8 W <= 256 every slot j of the order CR(n)
// holds at most one term, slot j = k, so the tree levels are: strides 4W, 2W
// and W pair c with c + 4, c + 2, c + 1 inside a lane; strides W/2 .. 1 pair
// lane g with lane g + s by an xor shuffle inside the group.  The levels run
// in the descending order of CR(n), skipping pairs whose upper slot holds no
// term, so the bits equal those of every other mapping.  Shuffles name only
// the group's lanes, so groups may take different branches.
#pragma once
#include "ngb_rowpath.cuh"

namespace ngb {

// The lanes of the group of `lane` (W = 8, 16 or 32).
template <int W>
__device__ __forceinline__ unsigned group_mask(int lane) {
  return W == 32 ? FULL : (((1u << W) - 1u) << (lane & ~(W - 1)));
}

// MagTrack reduced over the W lanes of a group.
template <int W>
__device__ __forceinline__ void group_reduce(MagTrack<float>& mt, unsigned gm) {
#pragma unroll
  for (int o = W / 2; o >= 1; o >>= 1) {
    mt.m = fmaxf(mt.m, __shfl_xor_sync(gm, mt.m, o));
    mt.nz = (__shfl_xor_sync(gm, mt.nz ? 1 : 0, o) != 0) || mt.nz;
  }
}
template <int W>
__device__ __forceinline__ void group_reduce(MagTrack<double>& mt, unsigned gm) {
#pragma unroll
  for (int o = W / 2; o >= 1; o >>= 1) {
    mt.k = max(mt.k, __shfl_xor_sync(gm, mt.k, o));
    mt.kmin1 = min(mt.kmin1, __shfl_xor_sync(gm, mt.kmin1, o));
  }
}

// The order CR(n) of the terms q (layout above) of one vector, n <= 8 W; the
// total is returned to every lane of the group (gbase: its first lane).
template <typename T, int W>
__device__ __forceinline__ T group_cr_tree(T (&q)[8], int n, int g, unsigned gm, int gbase) {
#pragma unroll
  for (int p = 4; p >= 1; p >>= 1) {
    if (n <= W * p) continue;  // no slot j < W p with a term at j + W p
#pragma unroll
    for (int c = 0; c < p; ++c)
      if (W * (c + p) + g < n) q[c] = FP<T>::add(q[c], q[c + p]);
  }
#pragma unroll
  for (int s = W / 2; s >= 1; s >>= 1) {
    const T o = __shfl_xor_sync(gm, q[0], s);
    if (g < s && g + s < n) q[0] = FP<T>::add(q[0], o);
  }
  return __shfl_sync(gm, q[0], gbase);
}

// Forward steps after the factor code is known: x~ = c x, the squares, the
// tree, r~ = sqrt, h = 1/r~, x^ = h x~ (EMU: binary64 integer-pipe scale,
// squares and a share of the outputs, as Chunk<double, 8, true>).
template <typename T, int W, bool EMU>
__device__ __forceinline__ void group_forward_tail(T (&v)[8], T* yr, int n, int g, unsigned gm, int gbase,
                                                   const VecOut<T>& out, int64_t vec, int code) {
  const T cf = factor_of<T, true>(code);
  if (code != CODE_ONE) Chunk<T, 8, EMU>::scale(cf, Pow2Scale<T>::exponent(code), v);
  T q[8];
  Chunk<T, 8, EMU>::squares(v, q);
  const T rt = FP<T>::sqrt(group_cr_tree<T, W>(q, n, g, gm, gbase));
  const T h = FP<T>::rcp(rt);
  if (yr) {
#pragma unroll
    for (int c = 0; c < 8; ++c)
      if (W * c + g < n) __stcs(yr + W * c + g, Chunk<T, 8, EMU>::template output<>(c, h, v[c]));
  }
  if (g == 0) out.put(vec, FP<T>::mul(inverse_of<T, true>(code), rt), h, code);
}

template <typename T, int W>
__device__ __forceinline__ void group_load(const T* __restrict__ xr, int n, int g, T (&v)[8]) {
#pragma unroll
  for (int c = 0; c < 8; ++c) v[c] = W * c + g < n ? __ldcs(xr + W * c + g) : T(0);
}

// A binary64 vector outside the range of the integer-pipe steps (rare): the
// hardware operations, out of line so that the common path stays small and
// its FP64 work is not predicated into the in-range path.
template <typename T, int W>
__device__ __noinline__ void group_forward_slow(const T* __restrict__ xr, T* yr, int n, int lane,
                                                const VecOut<T>& out, int64_t vec, int code) {
  const int g = lane & (W - 1);
  T v[8];
  group_load<T, W>(xr, n, g, v);
  group_forward_tail<T, W, false>(v, yr, n, g, group_mask<W>(lane), lane - g, out, vec, code);
}

// Forward of one vector of 5 <= n <= 8 W by the W lanes of the group of
// `lane`; yr may be null (norm only).  Every lane of the group calls it with
// the same arguments.
template <typename T, int W>
__device__ __forceinline__ void group_forward(const T* __restrict__ xr, T* yr, int n, int lane,
                                              const VecOut<T>& out, int64_t vec) {
  const int g = lane & (W - 1), gbase = lane - g;
  const unsigned gm = group_mask<W>(lane);
  T v[8];
  group_load<T, W>(xr, n, g, v);
  MagTrack<T> mt;
#pragma unroll
  for (int c = 0; c < 8; ++c) mt.take(v[c]);  // zero padding changes neither m nor the zero test
  group_reduce<W>(mt, gm);
  if (mt.zero()) {
    if (yr) {
#pragma unroll
      for (int c = 0; c < 8; ++c)
        if (W * c + g < n) __stcs(yr + W * c + g, T(0));
    }
    if (g == 0) out.put(vec, T(0), T(0), CODE_ZERO);
    return;
  }
  if (mt.has_nan()) {
    mt = MagTrack<T>();
#pragma unroll
    for (int c = 0; c < 8; ++c) mt.take_skip_nan(v[c]);
    group_reduce<W>(mt, gm);
  }
  const int code = mt.code();
  if (sizeof(T) == 8 && !mt.emu_ok(code)) {
    group_forward_slow<T, W>(xr, yr, n, lane, out, vec, code);
    return;
  }
  group_forward_tail<T, W, sizeof(T) == 8>(v, yr, n, g, gm, gbase, out, vec, code);
}

// Backward steps with the FP64 pipe's products: dot = CR(y_k g_k),
// grad_k = ((g_k - y_k dot) h) c, from y and g in registers.
template <typename T, int W>
__device__ __forceinline__ void group_backward_tail_hw(const T (&yv)[8], const T (&gv)[8], T* gradr, int n, int g,
                                                       unsigned gm, int gbase, T h, int code) {
  T q[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) q[c] = FP<T>::mul(yv[c], gv[c]);
  const T dot = group_cr_tree<T, W>(q, n, g, gm, gbase);
  const T cf = factor_of<T, true>(code);
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    if (W * c + g < n) {
      T o = FP<T>::mul(FP<T>::sub(gv[c], FP<T>::mul(yv[c], dot)), h);
      if (code != CODE_ONE) o = FP<T>::mul(o, cf);
      __stcs(gradr + W * c + g, o);
    }
  }
}

// The same for a binary64 vector whose products leave the integer-pipe
// range (rare): out of line, reading y and g again.
template <typename T, int W>
__device__ __noinline__ void group_backward_slow(const T* __restrict__ yr, const T* __restrict__ gr, T* gradr, int n,
                                                 int lane, T h, int code) {
  const int g = lane & (W - 1);
  T yv[8], gv[8];
  group_load<T, W>(yr, n, g, yv);
  group_load<T, W>(gr, n, g, gv);
  group_backward_tail_hw<T, W>(yv, gv, gradr, n, g, group_mask<W>(lane), lane - g, h, code);
}

// Backward of one vector of n <= 8 W by a group: dot = CR(y_k g_k),
// grad_k = ((g_k - y_k dot) h) c.  binary64 forms the products y_k g_k and
// y_k dot on the integer pipes (f64emu::mul_signed) when every one of them is
// in range, decided from the integer keys of y, g and dot (the same in every
// lane of the group); otherwise the out-of-line FP64 form redoes the vector.
// With c = 1, part of the products by h go to f64emu::mul as well when
// grad_h_in_range holds.  Every form gives the same bits.
template <typename T, int W>
__device__ __forceinline__ void group_backward(const T* __restrict__ yr, const T* __restrict__ gr, T* gradr, int n,
                                               int lane, T h, int code) {
  const int g = lane & (W - 1), gbase = lane - g;
  const unsigned gm = group_mask<W>(lane);
  if (code == CODE_ZERO) {
#pragma unroll
    for (int c = 0; c < 8; ++c)
      if (W * c + g < n) __stcs(gradr + W * c + g, T(0));
    return;
  }
  T yv[8], gv[8];
  group_load<T, W>(yr, n, g, yv);
  group_load<T, W>(gr, n, g, gv);
  if constexpr (sizeof(T) == 8) {
    MagTrack<double> ry, rg;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      ry.take(yv[c]);
      rg.take(gv[c]);
    }
    group_reduce<W>(ry, gm);
    group_reduce<W>(rg, gm);
    if (!products_in_range(ry, rg)) {
      group_backward_slow<T, W>(yr, gr, gradr, n, lane, h, code);
      return;
    }
    double q[8];
#pragma unroll
    for (int c = 0; c < 8; ++c)
      q[c] = __longlong_as_double(static_cast<long long>(f64emu::mul_signed(
          static_cast<uint64_t>(__double_as_longlong(yv[c])), static_cast<uint64_t>(__double_as_longlong(gv[c])))));
    const double dot = group_cr_tree<double, W>(q, n, g, gm, gbase);
    MagTrack<double> rd;
    rd.take(dot);
    if (!products_in_range(ry, rd)) {
      group_backward_slow<T, W>(yr, gr, gradr, n, lane, h, code);
      return;
    }
    const uint64_t db = static_cast<uint64_t>(__double_as_longlong(dot));
    // RN(g_k - RN(y_k dot)) RN-times h; with `hemu` the products by h of
    // chunks c < F64_EMU_GRAD_H_OF_8 by f64emu::mul and the differences of
    // chunks c >= 8 - F64_EMU_GRAD_SUB_OF_8 by f64emu::add_signed (see
    // grad_h_in_range)
    auto t = [&](int c, bool hemu) {
      const double p = __longlong_as_double(
          static_cast<long long>(f64emu::mul_signed(static_cast<uint64_t>(__double_as_longlong(yv[c])), db)));
      double d;
      if (hemu && c >= 8 - F64_EMU_GRAD_SUB_OF_8)
        d = __longlong_as_double(static_cast<long long>(
            f64emu::add_signed(static_cast<uint64_t>(__double_as_longlong(gv[c])),
                               static_cast<uint64_t>(__double_as_longlong(p)) ^ 0x8000000000000000ull)));
      else
        d = FP<double>::sub(gv[c], p);
      if (hemu && c < F64_EMU_GRAD_H_OF_8)
        return __longlong_as_double(static_cast<long long>(
            f64emu::mul(static_cast<uint64_t>(__double_as_longlong(d)), static_cast<uint64_t>(__double_as_longlong(h)))));
      return FP<double>::mul(d, h);
    };
    const bool hemu = F64_EMU_GRAD_H_OF_8 > 0 && grad_h_in_range(ry, rg, rd, h);  // group-uniform
    if (code != CODE_ONE) {  // group-uniform; the multiplication by c = 1 is skipped (exact)
      const double cf = factor_of<double, true>(code);
#pragma unroll
      for (int c = 0; c < 8; ++c)
        if (W * c + g < n) __stcs(gradr + W * c + g, FP<double>::mul(t(c, false), cf));
    } else if (hemu) {
#pragma unroll
      for (int c = 0; c < 8; ++c)
        if (W * c + g < n) __stcs(gradr + W * c + g, t(c, true));
    } else {
#pragma unroll
      for (int c = 0; c < 8; ++c)
        if (W * c + g < n) __stcs(gradr + W * c + g, t(c, false));
    }
  } else {
    group_backward_tail_hw<T, W>(yv, gv, gradr, n, g, gm, gbase, h, code);
  }
}

}  // namespace ngb
