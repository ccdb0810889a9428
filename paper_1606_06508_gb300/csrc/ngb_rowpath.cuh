// ngb_rowpath.cuh -- warp-per-vector and block-per-vector forms of the
// generic (n >= 5) scaling normalization and of its backward pass.
//
// The sum of squares (and the backward dot product) follows the canonical
// order CR(n): slot j < 256 is the left-to-right sum of terms j, j + 256, ...,
// then slot j <- slot j + slot (j + s) for s = 128, 64, ..., 1 whenever slot
// j + s holds a term.  Each mapping places the slots so that every tree level
// becomes either an in-register add, a warp shuffle (xor by a power of two)
// or one shared-memory exchange, and performs the levels in the same
// descending order, so thread, warp and block mappings give identical bits.
#pragma once
#include "ngb_arith.cuh"

namespace ngb {

constexpr unsigned FULL = 0xffffffffu;

template <typename T>
__device__ __forceinline__ T warp_fmax(T m) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) m = FP<T>::fmax(m, __shfl_xor_sync(FULL, m, o));
  return m;
}

// Streaming (evict-first) loads and stores of V consecutive elements.
template <typename T, int V> struct Vec;
template <typename T> struct Vec<T, 1> {
  __device__ __forceinline__ static void load(const T* p, T* v) { v[0] = __ldcs(p); }
  __device__ __forceinline__ static void store(T* p, const T* v) { __stcs(p, v[0]); }
};
template <> struct Vec<float, 4> {
  __device__ __forceinline__ static void load(const float* p, float* v) {
    float4 a = __ldcs(reinterpret_cast<const float4*>(p));
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  }
  __device__ __forceinline__ static void store(float* p, const float* v) {
    __stcs(reinterpret_cast<float4*>(p), make_float4(v[0], v[1], v[2], v[3]));
  }
};
template <> struct Vec<double, 2> {
  __device__ __forceinline__ static void load(const double* p, double* v) {
    double2 a = __ldcs(reinterpret_cast<const double2*>(p));
    v[0] = a.x; v[1] = a.y;
  }
  __device__ __forceinline__ static void store(double* p, const double* v) {
    __stcs(reinterpret_cast<double2*>(p), make_double2(v[0], v[1]));
  }
};

// ---------------------------------------------------------------------------
// Warp layout (row held in registers).  Lane l holds chunk c (c < CH) as the
// V elements k = 32 V c + V l + e, e < V.  Slot j = k mod 256, so with
// G = 256/(32V) chunk groups: strides >= 32V pair chunk c with c + s/(32V)
// inside a lane, strides V .. 16V pair lane l with lane l ^ (s/V), and strides
// < V pair element e with e + s inside a lane.  Chunks c >= G are added in
// ascending order into the accumulator of chunk c mod G.
// Requires n <= 32 V CH; for V > 1 also n % V == 0 and 16-byte aligned rows.
template <typename T, int V, int CH>
__device__ __forceinline__ T warp_cr_tree(T (&q)[CH][V], int n, int lane) {
  constexpr int G = CR_SLOTS / (32 * V);
  constexpr int NS = CH < G ? CH : G;
  const int used = n < CR_SLOTS ? n : CR_SLOTS;
  // slots with more than one term: sequential adds in ascending k
#pragma unroll
  for (int c = G; c < CH; ++c) {
#pragma unroll
    for (int e = 0; e < V; ++e)
      if (32 * V * c + V * lane + e < n) q[c % G][e] = FP<T>::add(q[c % G][e], q[c][e]);
  }
  // strides 128 .. 32V: chunk c += chunk c + p
#pragma unroll
  for (int p = G / 2; p >= 1; p >>= 1) {
#pragma unroll
    for (int c = 0; c < p; ++c) {
      if (c + p < NS) {
#pragma unroll
        for (int e = 0; e < V; ++e)
          if (32 * V * (c + p) + V * lane + e < used) q[c][e] = FP<T>::add(q[c][e], q[c + p][e]);
      }
    }
  }
  // strides 16V .. V: lane l += lane l + p.  When every slot holds a term the
  // level is a butterfly on all lanes: lane l and lane l ^ p both form the
  // same sum (addition is commutative), so no lane needs a predicate.
  if (used == CR_SLOTS) {
#pragma unroll
    for (int p = 16; p >= 1; p >>= 1) {
#pragma unroll
      for (int e = 0; e < V; ++e) q[0][e] = FP<T>::add(q[0][e], __shfl_xor_sync(FULL, q[0][e], p));
    }
  } else {
#pragma unroll
    for (int p = 16; p >= 1; p >>= 1) {
#pragma unroll
      for (int e = 0; e < V; ++e) {
        const T o = __shfl_xor_sync(FULL, q[0][e], p);
        if (lane < p && V * (lane + p) + e < used) q[0][e] = FP<T>::add(q[0][e], o);
      }
    }
  }
  // strides V/2 .. 1 inside lane 0
#pragma unroll
  for (int p = V / 2; p >= 1; p >>= 1) {
#pragma unroll
    for (int e = 0; e < p; ++e)
      if (e + p < used) q[0][e] = FP<T>::add(q[0][e], q[0][e + p]);
  }
  if (used == CR_SLOTS) return q[0][0];  // the butterfly left the total in every lane
  return __shfl_sync(FULL, q[0][0], 0);
}

// Forward of a binary32 vector of 5 <= n <= 64 CH by one half-warp (16 lanes,
// gmask names them): lane hl holds the float4 chunks k = 64 c + 4 hl, i.e. the
// CR slots 64 c + 4 hl + e.  Tree: strides 128 and 64 across the lane's
// chunks, 32 .. 4 by shuffles inside the half-warp (offsets 8 .. 1), 2 and 1
// inside the float4.  Two vectors per warp: half the shuffle levels per
// vector of the 32-lane layout, and twice the loads in flight per warp.
// xr must be 16-byte aligned and n a multiple of 4.
template <int CH>
__device__ __forceinline__ void half_forward_f32(const float* __restrict__ xr, float* yr, int n, int hl,
                                                 unsigned gmask, const VecOut<float>& out, int64_t vec, bool put) {
  float v[CH][4];
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const int k0 = 64 * c + 4 * hl;
    if (k0 < n) {
      Vec<float, 4>::load(xr + k0, v[c]);
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) v[c][e] = 0.0f;
    }
  }
  float m = 0.0f;
  bool nz = false;
#pragma unroll
  for (int c = 0; c < CH; ++c) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      nz |= !(v[c][e] == 0.0f);
      m = fmaxf(m, fabsf(v[c][e]));
    }
  }
#pragma unroll
  for (int o = 8; o >= 1; o >>= 1) m = fmaxf(m, __shfl_xor_sync(gmask, m, o));
  nz = (__ballot_sync(gmask, nz) & gmask) != 0u;
  if (!nz) {
    if (yr) {
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        const int k0 = 64 * c + 4 * hl;
        const float z[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        if (k0 < n) Vec<float, 4>::store(yr + k0, z);
      }
    }
    if (put && hl == 0) out.put(vec, 0.0f, 0.0f, CODE_ZERO);
    return;
  }
  const int code = select_code<float, true>(m);
  const float cf = factor_of<float, true>(code);
  if (code != CODE_ONE) {
#pragma unroll
    for (int c = 0; c < CH; ++c) {
#pragma unroll
      for (int e = 0; e < 4; ++e) v[c][e] = __fmul_rn(cf, v[c][e]);
    }
  }
  float q[CH][4];
#pragma unroll
  for (int c = 0; c < CH; ++c) {
#pragma unroll
    for (int e = 0; e < 4; ++e) q[c][e] = __fmul_rn(v[c][e], v[c][e]);
  }
  const int used = n < CR_SLOTS ? n : CR_SLOTS;
  // strides 128 .. 64: chunk c += chunk c + p
#pragma unroll
  for (int p = CH / 2; p >= 1; p >>= 1) {
#pragma unroll
    for (int c = 0; c < p; ++c) {
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (64 * (c + p) + 4 * hl + e < used) q[c][e] = __fadd_rn(q[c][e], q[c + p][e]);
    }
  }
  // strides 32 .. 4: lane hl += lane hl + p (butterfly when every slot holds a term)
  if (used == 64 * CH && used == CR_SLOTS) {
#pragma unroll
    for (int p = 8; p >= 1; p >>= 1) {
#pragma unroll
      for (int e = 0; e < 4; ++e) q[0][e] = __fadd_rn(q[0][e], __shfl_xor_sync(gmask, q[0][e], p));
    }
  } else {
#pragma unroll
    for (int p = 8; p >= 1; p >>= 1) {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float o = __shfl_xor_sync(gmask, q[0][e], p);
        if (hl < p && 4 * (hl + p) + e < used) q[0][e] = __fadd_rn(q[0][e], o);
      }
    }
  }
  // strides 2, 1 inside the float4
#pragma unroll
  for (int p = 2; p >= 1; p >>= 1) {
#pragma unroll
    for (int e = 0; e < p; ++e)
      if (e + p < used) q[0][e] = __fadd_rn(q[0][e], q[0][e + p]);
  }
  const int src = (int)(__ffs(gmask) - 1);  // lane 0 of the half-warp
  const float total = (used == CR_SLOTS) ? q[0][0] : __shfl_sync(gmask, q[0][0], src);
  const float rt = __fsqrt_rn(total);
  const float h = __frcp_rn(rt);
  if (yr) {
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      const int k0 = 64 * c + 4 * hl;
      if (k0 < n) {
        float o[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) o[e] = __fmul_rn(h, v[c][e]);
        Vec<float, 4>::store(yr + k0, o);
      }
    }
  }
  if (put && hl == 0) out.put(vec, __fmul_rn(inverse_of<float, true>(code), rt), h, code);
}

// Backward, one warp per vector: dot = CR(y_k g_k), grad_k = ((g_k - y_k dot) h) c.
template <typename T, int V, int CH>
__device__ __forceinline__ void warp_backward(const T* __restrict__ yr, const T* __restrict__ gr, T* gradr, int n,
                                              int lane, T h, int code) {
  if (code == CODE_ZERO) {
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      const int k0 = 32 * V * c + V * lane;
      T z[V];
#pragma unroll
      for (int e = 0; e < V; ++e) z[e] = T(0);
      if (k0 < n) Vec<T, V>::store(gradr + k0, z);
    }
    return;
  }
  const T cf = factor_of<T, true>(code);
  T yv[CH][V], gv[CH][V], q[CH][V];
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const int k0 = 32 * V * c + V * lane;
    if (k0 < n) {
      Vec<T, V>::load(yr + k0, yv[c]);
      Vec<T, V>::load(gr + k0, gv[c]);
    } else {
#pragma unroll
      for (int e = 0; e < V; ++e) { yv[c][e] = T(0); gv[c][e] = T(0); }
    }
#pragma unroll
    for (int e = 0; e < V; ++e) q[c][e] = FP<T>::mul(yv[c][e], gv[c][e]);
  }
  const T dot = warp_cr_tree<T, V, CH>(q, n, lane);
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const int k0 = 32 * V * c + V * lane;
    if (k0 < n) {
      T o[V];
#pragma unroll
      for (int e = 0; e < V; ++e)
        o[e] = FP<T>::mul(FP<T>::mul(FP<T>::sub(gv[c][e], FP<T>::mul(yv[c][e], dot)), h), cf);
      Vec<T, V>::store(gradr + k0, o);
    }
  }
}

// ---------------------------------------------------------------------------
// Block layout (B threads, B = 64, 128 or 256).  Thread t holds the elements
// k = B c + t.  Slot j = k mod 256 belongs to thread j mod B, as its
// accumulator j / B (G = 256 / B of them): strides >= B are in-thread, the
// remaining strides B/2 .. 1 run in warp 0 after one pass through shared
// memory (lane l takes slots l + 32 i: strides B/2 .. 32 in-lane, then
// shuffles 16 .. 1).
template <typename T, int B>
struct BlockShared {
  T slot[B];
  T red[B / 32];
  T total;
  uint32_t kred[B / 32];
  int item;
  int flag;
};

template <typename T, int B>
__device__ __forceinline__ T block_fmax(T m, BlockShared<T, B>& sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  m = warp_fmax(m);
  if (lane == 0) sh.red[w] = m;
  __syncthreads();
  if (w == 0) {
    T a = lane < B / 32 ? sh.red[lane] : T(0);
    a = warp_fmax(a);
    if (lane == 0) sh.total = a;
  }
  __syncthreads();
  const T r = sh.total;
  __syncthreads();
  return r;
}

// MagTrack over the block; every thread gets the result.
template <int B>
__device__ __forceinline__ void block_reduce_mag(MagTrack<float>& mt, BlockShared<float, B>& sh) {
  mt.nz = __syncthreads_or(mt.nz);
  mt.m = block_fmax<float, B>(mt.m, sh);
}
template <int B>
__device__ __forceinline__ void block_reduce_mag(MagTrack<double>& mt, BlockShared<double, B>& sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t k = __reduce_max_sync(FULL, mt.k);
  if (lane == 0) sh.kred[w] = k;
  __syncthreads();
  uint32_t r = sh.kred[0];
#pragma unroll
  for (int i = 1; i < B / 32; ++i) r = max(r, sh.kred[i]);
  __syncthreads();
  mt.k = r;
}

// acc[i] holds slot i B + t of thread t (strides >= B already applied by the
// caller).  Returns the CR(n) total to every thread.
template <typename T, int B>
__device__ __forceinline__ T block_cr_finish(T acc0, int used, BlockShared<T, B>& sh) {
  const int t = threadIdx.x;
  sh.slot[t] = acc0;
  __syncthreads();
  if (t < 32) {
    constexpr int Q = B / 32;
    T a[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) a[i] = sh.slot[t + 32 * i];
#pragma unroll
    for (int p = Q / 2; p >= 1; p >>= 1) {
#pragma unroll
      for (int i = 0; i < p; ++i)
        if (32 * (i + p) + t < used) a[i] = FP<T>::add(a[i], a[i + p]);
    }
#pragma unroll
    for (int p = 16; p >= 1; p >>= 1) {
      const T o = __shfl_xor_sync(FULL, a[0], p);
      if (t < p && t + p < used) a[0] = FP<T>::add(a[0], o);
    }
    if (t == 0) sh.total = a[0];
  }
  __syncthreads();
  const T r = sh.total;
  __syncthreads();
  return r;
}

// In-thread part of the tree: accumulators of chunk c (c < CH) into slot
// group c mod G, then strides 128 .. B.
template <typename T, int B, int CH>
__device__ __forceinline__ T block_cr_tree(T (&q)[CH], int n, BlockShared<T, B>& sh) {
  constexpr int G = CR_SLOTS / B;
  constexpr int NS = CH < G ? CH : G;
  const int t = threadIdx.x;
  const int used = n < CR_SLOTS ? n : CR_SLOTS;
#pragma unroll
  for (int c = G; c < CH; ++c)
    if (B * c + t < n) q[c % G] = FP<T>::add(q[c % G], q[c]);
#pragma unroll
  for (int p = G / 2; p >= 1; p >>= 1) {
#pragma unroll
    for (int i = 0; i < p; ++i)
      if (i + p < NS && B * (i + p) + t < used) q[i] = FP<T>::add(q[i], q[i + p]);
  }
  return block_cr_finish<T, B>(q[0], used, sh);
}

// Forward, one block per vector held in registers (n <= B CH).
template <typename T, int B, int CH>
__device__ __forceinline__ void block_forward(const T* __restrict__ xr, T* yr, int n, const VecOut<T>& out,
                                              int64_t vec, BlockShared<T, B>& sh) {
  const int t = threadIdx.x;
  T v[CH];
  MagTrack<T> mt;
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const int k = B * c + t;
    v[c] = k < n ? __ldcs(xr + k) : T(0);
    mt.take(v[c]);
  }
  block_reduce_mag<B>(mt, sh);
  if (mt.zero()) {
    if (yr) {
#pragma unroll
      for (int c = 0; c < CH; ++c)
        if (B * c + t < n) __stcs(yr + B * c + t, T(0));
    }
    if (t == 0) out.put(vec, T(0), T(0), CODE_ZERO);
    return;
  }
  if (mt.has_nan()) {
    mt = MagTrack<T>();
#pragma unroll
    for (int c = 0; c < CH; ++c) mt.take_skip_nan(v[c]);
    block_reduce_mag<B>(mt, sh);
  }
  const int code = mt.code();
  const T cf = factor_of<T, true>(code);
  T q[CH];
  if (code != CODE_ONE) Chunk<T, CH, false>::scale(cf, Pow2Scale<T>::exponent(code), v);
  Chunk<T, CH, false>::squares(v, q);
  const T rt = FP<T>::sqrt(block_cr_tree<T, B, CH>(q, n, sh));
  const T h = FP<T>::rcp(rt);
  if (yr) {
#pragma unroll
    for (int c = 0; c < CH; ++c)
      if (B * c + t < n) __stcs(yr + B * c + t, FP<T>::mul(h, v[c]));
  }
  if (t == 0) out.put(vec, FP<T>::mul(inverse_of<T, true>(code), rt), h, code);
}

// Forward, one block per vector of any length up to 2^20: three passes over
// the row (largest magnitude, sum of squares, outputs); the second and third
// usually hit L2.
template <typename T, int B>
__device__ __forceinline__ void block_forward_stream(const T* __restrict__ xr, T* yr, int n, const VecOut<T>& out,
                                                     int64_t vec, BlockShared<T, B>& sh) {
  constexpr int G = CR_SLOTS / B;
  const int t = threadIdx.x;
  MagTrack<T> mt;
  for (int k = t; k < n; k += B) mt.take(xr[k]);
  block_reduce_mag<B>(mt, sh);
  if (mt.zero()) {
    if (yr)
      for (int k = t; k < n; k += B) yr[k] = T(0);
    if (t == 0) out.put(vec, T(0), T(0), CODE_ZERO);
    return;
  }
  if (mt.has_nan()) {
    mt = MagTrack<T>();
    for (int k = t; k < n; k += B) mt.take_skip_nan(xr[k]);
    block_reduce_mag<B>(mt, sh);
  }
  const int code = mt.code();
  const T cf = factor_of<T, true>(code);
  const int E = Pow2Scale<T>::exponent(code);
  T acc[G];
  {
    T a[G];
#pragma unroll
    for (int i = 0; i < G; ++i) {
      const int k = B * i + t;
      a[i] = k < n ? xr[k] : T(0);
    }
    if (code != CODE_ONE) Chunk<T, G, false>::scale(cf, E, a);
    Chunk<T, G, false>::squares(a, acc);
  }
  for (int base = CR_SLOTS; base < n; base += CR_SLOTS) {
    T a[G], q[G];
#pragma unroll
    for (int i = 0; i < G; ++i) {
      const int k = base + B * i + t;
      a[i] = k < n ? xr[k] : T(0);
    }
    if (code != CODE_ONE) Chunk<T, G, false>::scale(cf, E, a);
    Chunk<T, G, false>::squares(a, q);
#pragma unroll
    for (int i = 0; i < G; ++i)
      if (base + B * i + t < n) acc[i] = FP<T>::add(acc[i], q[i]);
  }
  const int used = n < CR_SLOTS ? n : CR_SLOTS;
#pragma unroll
  for (int p = G / 2; p >= 1; p >>= 1) {
#pragma unroll
    for (int i = 0; i < p; ++i)
      if (B * (i + p) + t < used) acc[i] = FP<T>::add(acc[i], acc[i + p]);
  }
  const T rt = FP<T>::sqrt(block_cr_finish<T, B>(acc[0], used, sh));
  const T h = FP<T>::rcp(rt);
  if (yr) {
    for (int k = t; k < n; k += B) {
      T a[1] = {xr[k]};
      if (code != CODE_ONE) Chunk<T, 1, false>::scale(cf, E, a);
      yr[k] = FP<T>::mul(h, a[0]);
    }
  }
  if (t == 0) out.put(vec, FP<T>::mul(inverse_of<T, true>(code), rt), h, code);
}

// Backward, one block per vector held in registers (n <= B CH).
template <typename T, int B, int CH>
__device__ __forceinline__ void block_backward(const T* __restrict__ yr, const T* __restrict__ gr, T* gradr, int n,
                                               T h, int code, BlockShared<T, B>& sh) {
  const int t = threadIdx.x;
  if (code == CODE_ZERO) {
#pragma unroll
    for (int c = 0; c < CH; ++c)
      if (B * c + t < n) __stcs(gradr + B * c + t, T(0));
    return;
  }
  const T cf = factor_of<T, true>(code);
  T yv[CH], gv[CH], q[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const int k = B * c + t;
    yv[c] = k < n ? __ldcs(yr + k) : T(0);
    gv[c] = k < n ? __ldcs(gr + k) : T(0);
    q[c] = FP<T>::mul(yv[c], gv[c]);
  }
  const T dot = block_cr_tree<T, B, CH>(q, n, sh);
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const int k = B * c + t;
    if (k < n) __stcs(gradr + k, FP<T>::mul(FP<T>::mul(FP<T>::sub(gv[c], FP<T>::mul(yv[c], dot)), h), cf));
  }
}

// Backward, one block per vector of any length (two passes over y and g).
template <typename T, int B>
__device__ __forceinline__ void block_backward_stream(const T* __restrict__ yr, const T* __restrict__ gr, T* gradr,
                                                      int n, T h, int code, BlockShared<T, B>& sh) {
  constexpr int G = CR_SLOTS / B;
  const int t = threadIdx.x;
  if (code == CODE_ZERO) {
    for (int k = t; k < n; k += B) gradr[k] = T(0);
    return;
  }
  const T cf = factor_of<T, true>(code);
  T acc[G];
#pragma unroll
  for (int i = 0; i < G; ++i) {
    const int k = B * i + t;
    acc[i] = k < n ? FP<T>::mul(yr[k], gr[k]) : T(0);
  }
  for (int base = CR_SLOTS; base < n; base += CR_SLOTS) {
#pragma unroll
    for (int i = 0; i < G; ++i) {
      const int k = base + B * i + t;
      if (k < n) acc[i] = FP<T>::add(acc[i], FP<T>::mul(yr[k], gr[k]));
    }
  }
  const int used = n < CR_SLOTS ? n : CR_SLOTS;
#pragma unroll
  for (int p = G / 2; p >= 1; p >>= 1) {
#pragma unroll
    for (int i = 0; i < p; ++i)
      if (B * (i + p) + t < used) acc[i] = FP<T>::add(acc[i], acc[i + p]);
  }
  const T dot = block_cr_finish<T, B>(acc[0], used, sh);
  for (int k = t; k < n; k += B)
    gradr[k] = FP<T>::mul(FP<T>::mul(FP<T>::sub(gr[k], FP<T>::mul(yr[k], dot)), h), cf);
}

// ---------------------------------------------------------------------------
// Rounds of 8 loads per lane that a binary32 streaming pass keeps in flight
// (ragged binary32 workload, fraction of the copy bandwidth: 2 rounds 0.870,
// 3 rounds 0.877 at the same 48 registers; 4 and 8 spill and run slower).
constexpr int STREAM_ROUNDS = 3;

// Streaming warp layout (any length).  Lane l reads the elements
// k = 32 c + l, c = 0, 1, ..., eight chunks (256 elements) per round; slot
// k mod 256 = 32 (c mod 8) + l is lane l's partial sum acc[c mod 8],
// accumulated in ascending c.  Tree: strides 128, 64, 32 inside the lane,
// 16 .. 1 by shuffles.  Nothing of the vector is held between passes: each
// pass reads it again (the second and third reads usually hit L2).
// The in-lane levels (strides 128, 64, 32): lane l's partial sum of slot l.
template <typename T>
__device__ __forceinline__ T stream_tree_lane(T (&acc)[8], int n, int lane) {
  const int used = n < CR_SLOTS ? n : CR_SLOTS;
#pragma unroll
  for (int p = 4; p >= 1; p >>= 1) {
    if (used <= 32 * p) continue;  // warp-uniform: no slot of chunks p .. 2p-1 holds a term
#pragma unroll
    for (int i = 0; i < p; ++i)
      if (32 * (i + p) + lane < used) acc[i] = FP<T>::add(acc[i], acc[i + p]);
  }
  return acc[0];
}

// The shuffle levels (strides 16 .. 1) on the lane partials v; the total is
// returned to every lane.
template <typename T>
__device__ __forceinline__ T stream_tree_shfl(T v, int n, int lane) {
  const int used = n < CR_SLOTS ? n : CR_SLOTS;
  if (used == CR_SLOTS) {  // butterfly: every lane ends with the total
#pragma unroll
    for (int p = 16; p >= 1; p >>= 1) v = FP<T>::add(v, __shfl_xor_sync(FULL, v, p));
    return v;
  }
#pragma unroll
  for (int p = 16; p >= 1; p >>= 1) {
    const T o = __shfl_xor_sync(FULL, v, p);
    if (lane < p && lane + p < used) v = FP<T>::add(v, o);
  }
  return __shfl_sync(FULL, v, 0);
}

// The shuffle levels for two vectors at once: a and b are the lane partials
// of vectors A (na components) and B (nb).  The first exchange leaves slot
// i + 16 added into slot i of A in lane i and of B in lane 16 + i (i < 16);
// the remaining levels run inside each half-warp and serve both vectors with
// one instruction.  The additions and their order are those of CR(n) for each
// vector.  Returns A's total in lane 0 and B's in lane 16.
// Stride 16 of stream_tree_shfl2: slot i (i < 16) of A in lane i, of B in
// lane 16 + i.
template <typename T>
__device__ __forceinline__ T stream_tree_shfl2_level16(T a, int na, T b, int nb, int lane) {
  const bool hi = lane >= 16;
  const int i = lane & 15;
  const int used = hi ? (nb < CR_SLOTS ? nb : CR_SLOTS) : (na < CR_SLOTS ? na : CR_SLOTS);
  const T o16 = __shfl_xor_sync(FULL, hi ? a : b, 16);  // lane i gets A's slot i + 16, lane 16 + i B's slot i
  // lane 16 + i holds B's slot 16 + i itself: added to slot i when it holds a
  // term, otherwise slot i alone moves there
  T r = hi ? b : a;
  if (i + 16 < used) r = FP<T>::add(r, o16);
  else if (hi) r = o16;
  return r;
}

template <typename T>
__device__ __forceinline__ T stream_tree_shfl2(T a, int na, T b, int nb, int lane) {
  const bool hi = lane >= 16;
  const int i = lane & 15;
  const int used = hi ? (nb < CR_SLOTS ? nb : CR_SLOTS) : (na < CR_SLOTS ? na : CR_SLOTS);
  T r = stream_tree_shfl2_level16<T>(a, na, b, nb, lane);
#pragma unroll
  for (int p = 8; p >= 1; p >>= 1) {
    const T o = __shfl_xor_sync(FULL, r, p);
    if (i < p && i + p < used) r = FP<T>::add(r, o);
  }
  return r;
}

// The same for four vectors A, B, C, D (lane partials a, b, c, d; lengths
// na .. nd).  Stride 16 as in stream_tree_shfl2, once for (A, B) and once for
// (C, D); stride 8 then exchanges between the two: in each half-warp, lanes
// i < 8 add slot i + 8 into slot i of A (or B), lanes i >= 8 slot i into
// slot i - 8 of C (or D), so that each quarter-warp holds the first 8 slots
// of one vector (lanes 0-7 A, 8-15 C, 16-23 B, 24-31 D) for strides 4, 2, 1.
// Returns the totals in lanes 0 (A), 16 (B), 8 (C) and 24 (D).
template <typename T>
__device__ __forceinline__ T stream_tree_shfl4(T a, int na, T b, int nb, T c, int nc, T d, int nd, int lane) {
  const T r1 = stream_tree_shfl2_level16<T>(a, na, b, nb, lane);
  const T r2 = stream_tree_shfl2_level16<T>(c, nc, d, nd, lane);
  const bool hi = lane >= 16;
  const int i = lane & 15;
  const bool lo8 = i < 8;
  const int nv = lo8 ? (hi ? nb : na) : (hi ? nd : nc);
  const int used = nv < CR_SLOTS ? nv : CR_SLOTS;
  const T o8 = __shfl_xor_sync(FULL, lo8 ? r2 : r1, 8);
  const int j = i & 7;  // the slot this lane holds after the exchange
  T r = lo8 ? r1 : r2;
  if (j + 8 < used) r = FP<T>::add(r, o8);
#pragma unroll
  for (int p = 4; p >= 1; p >>= 1) {
    const T o = __shfl_xor_sync(FULL, r, p);
    if (j < p && j + p < used) r = FP<T>::add(r, o);
  }
  return r;
}

template <typename T>
__device__ __forceinline__ T stream_tree(T (&acc)[8], int n, int lane) {
  return stream_tree_shfl<T>(stream_tree_lane<T>(acc, n, lane), n, lane);
}

// Eight chunks of one round; rounds that lie inside the vector skip the
// per-element bounds test.
template <typename T>
__device__ __forceinline__ void stream_load8(const T* __restrict__ p, int base, int n, int lane, T (&v)[8]) {
  if (base + 256 <= n) {
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = p[base + 32 * i + lane];
  } else {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int k = base + 32 * i + lane;
      v[i] = k < n ? p[k] : T(0);
    }
  }
}

// Pass 2 of the forward: the scaled squares in the order CR(n).  SCALED
// selects x~ = c x; otherwise x~ = x (c = 1).
// LANE: return lane l's partial sum after the in-lane levels only (the
// shuffle levels left to the caller, stream_tree_shfl2).
template <typename T, bool SCALED, bool EMU, bool TAIL_SKIP = true, bool LANE = false>
__device__ __forceinline__ T stream_sum_squares(const T* __restrict__ xr, int n, int lane, T cf, int E) {
  T acc[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) acc[i] = T(0);
  {  // first round: one term per slot (slots beyond n are never read by the tree)
    T v[8];
    stream_load8(xr, 0, n, lane, v);
    if (SCALED) Chunk<T, 8, EMU>::scale(cf, E, v);
    Chunk<T, 8, EMU>::squares(v, acc);
  }
  int base = 256;
  for (; base + 256 <= n; base += 256) {  // full rounds
    T v[8], q[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = xr[base + 32 * i + lane];
    if (SCALED) Chunk<T, 8, EMU>::scale(cf, E, v);
    Chunk<T, 8, EMU>::squares(v, q);
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i] = FP<T>::add(acc[i], q[i]);
  }
  if (base < n) {  // last, partial round
    T v[8], q[8];
    stream_load8(xr, base, n, lane, v);
    if (SCALED) Chunk<T, 8, EMU>::scale(cf, E, v);
    Chunk<T, 8, EMU>::squares(v, q);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if (TAIL_SKIP && base + 32 * i >= n) break;  // warp-uniform: no additions for chunks past the end
      if (base + 32 * i + lane < n) acc[i] = FP<T>::add(acc[i], q[i]);
    }
  }
  if (LANE) return stream_tree_lane<T>(acc, n, lane);
  return stream_tree<T>(acc, n, lane);
}

// Pass 3 of the forward: x^ = h x~, written with evict-first stores.
template <typename T, bool SCALED, bool EMU, int OUTK = F64_EMU_OUTPUTS_OF_8>
__device__ __forceinline__ void stream_write(const T* __restrict__ xr, T* yr, int n, int lane, T h, T cf, int E) {
  int base = 0;
  if (sizeof(T) == 4) {  // binary32: STREAM_ROUNDS rounds of loads in flight
    constexpr int R = STREAM_ROUNDS;
    for (; base + 256 * R <= n; base += 256 * R) {
      T v[R][8];
#pragma unroll
      for (int r = 0; r < R; ++r) {
#pragma unroll
        for (int i = 0; i < 8; ++i) v[r][i] = __ldcs(xr + base + 256 * r + 32 * i + lane);
      }
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (SCALED) Chunk<T, 8, EMU>::scale(cf, E, v[r]);
#pragma unroll
        for (int i = 0; i < 8; ++i)
          __stcs(yr + base + 256 * r + 32 * i + lane, Chunk<T, 8, EMU>::template output<OUTK>(i, h, v[r][i]));
      }
    }
  }
  for (; base + 256 <= n; base += 256) {
    T v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __ldcs(xr + base + 32 * i + lane);
    if (SCALED) Chunk<T, 8, EMU>::scale(cf, E, v);
#pragma unroll
    for (int i = 0; i < 8; ++i) __stcs(yr + base + 32 * i + lane, Chunk<T, 8, EMU>::template output<OUTK>(i, h, v[i]));
  }
  if (base < n) {
    T v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int k = base + 32 * i + lane;
      v[i] = k < n ? __ldcs(xr + k) : T(0);
    }
    if (SCALED) Chunk<T, 8, EMU>::scale(cf, E, v);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if (base + 32 * i >= n) break;  // warp-uniform: no work for chunks past the end
      const int k = base + 32 * i + lane;
      if (k < n) __stcs(yr + k, Chunk<T, 8, EMU>::template output<OUTK>(i, h, v[i]));
    }
  }
}

// Pass 1 of the streaming forward: the largest magnitude and the zero test.
// binary32 also runs pass 2 speculatively, for the factor c0 that the largest
// magnitude of the first round (the first 256 components) selects: the sum of
// squares of c0 x in the order CR(n), which saves the second pass whenever the
// whole vector selects the same factor (always for n <= 256; measured on the
// 4e6-vector ragged binary32 workload, where about half of the vectors need
// scaling: 0.870 of the copy bandwidth against 0.845 when speculating on
// c = 1 only).  The speculative terms are formed exactly as pass 2 forms
// them, so the bits are the same.  binary64 does not speculate: there
// the squares are integer-pipe work that would slow this first, HBM-bound
// pass (measured: 15 % slower on the ragged binary64 workload).  For a zero
// vector it writes the zero result and returns CODE_ZERO.  Otherwise it
// returns the factor code and sets `emu` when the integer-pipe steps take
// every component; `s` is the algorithm's sum of squares when `have_s`.  When
// the speculation fails (another factor) the caller runs pass 2 and the
// speculative sum, possibly overflowed, is discarded unread.
template <typename T>
__device__ __forceinline__ int stream_pass1(const T* __restrict__ xr, T* yr, int n, int lane, const VecOut<T>& out,
                                            int64_t vec, bool& emu, T& s, bool& have_s) {
  constexpr bool SPEC = sizeof(T) == 4;
  MagTrack<T> mt;
  T acc[8];
  int code0 = CODE_ONE;
  T cf0 = T(1);
  int E0 = 0;
  {
    T v[8];
    stream_load8(xr, 0, n, lane, v);
#pragma unroll
    for (int i = 0; i < 8; ++i) mt.take(v[i]);  // zero padding changes neither m nor the zero test
    if (SPEC) {
      MagTrack<T> m0 = mt;
      m0.warp_reduce();
      if (!m0.zero()) code0 = m0.code();
      if (code0 != CODE_ONE) {
        cf0 = factor_of<T, true>(code0);
        E0 = Pow2Scale<T>::exponent(code0);
        Chunk<T, 8, false>::scale(cf0, E0, v);
      }
      Chunk<T, 8, false>::squares(v, acc);
    }
  }
  int base = 256;
  // binary32: STREAM_ROUNDS rounds (8 loads per lane each) in flight per
  // iteration, taken in ascending order, so the slot sums are unchanged
  constexpr int R = sizeof(T) == 4 ? STREAM_ROUNDS : 1;
  for (; base + 256 * R <= n; base += 256 * R) {
    T v[R][8];
#pragma unroll
    for (int r = 0; r < R; ++r) {
#pragma unroll
      for (int i = 0; i < 8; ++i) v[r][i] = xr[base + 256 * r + 32 * i + lane];
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      T q[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) mt.take(v[r][i]);
      if (SPEC) {
        if (code0 != CODE_ONE) Chunk<T, 8, false>::scale(cf0, E0, v[r]);
        Chunk<T, 8, false>::squares(v[r], q);
#pragma unroll
        for (int i = 0; i < 8; ++i) acc[i] = FP<T>::add(acc[i], q[i]);
      }
    }
  }
  for (; base + 256 <= n; base += 256) {
    T v[8], q[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = xr[base + 32 * i + lane];
#pragma unroll
    for (int i = 0; i < 8; ++i) mt.take(v[i]);
    if (SPEC) {
      if (code0 != CODE_ONE) Chunk<T, 8, false>::scale(cf0, E0, v);
      Chunk<T, 8, false>::squares(v, q);
#pragma unroll
      for (int i = 0; i < 8; ++i) acc[i] = FP<T>::add(acc[i], q[i]);
    }
  }
  if (base < n) {
    T v[8], q[8];
    stream_load8(xr, base, n, lane, v);
#pragma unroll
    for (int i = 0; i < 8; ++i) mt.take(v[i]);
    if (SPEC) {
      if (code0 != CODE_ONE) Chunk<T, 8, false>::scale(cf0, E0, v);
      Chunk<T, 8, false>::squares(v, q);
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if (base + 32 * i + lane < n) acc[i] = FP<T>::add(acc[i], q[i]);
    }
  }
  mt.warp_reduce();
  if (mt.zero()) {
    if (yr)
      for (int k = lane; k < n; k += 32) __stcs(yr + k, T(0));
    if (lane == 0) out.put(vec, T(0), T(0), CODE_ZERO);
    emu = false;
    have_s = false;
    return CODE_ZERO;
  }
  if (mt.has_nan()) {
    mt = MagTrack<T>();
    for (int k = lane; k < n; k += 32) mt.take_skip_nan(xr[k]);
    mt.warp_reduce();
  }
  const int code = mt.code();
  emu = mt.emu_ok(code);
  have_s = SPEC && code == code0;
  s = SPEC ? stream_tree<T>(acc, n, lane) : T(0);
  return code;
}

// Pass 2 for a vector with factor code `code` (not CODE_ZERO); EMU selects
// the binary64 integer-pipe steps.
template <typename T, bool EMU, bool TAIL_SKIP = true, bool LANE = false>
__device__ __forceinline__ T stream_pass2(const T* __restrict__ xr, int n, int lane, int code) {
  const T cf = factor_of<T, true>(code);
  const int E = Pow2Scale<T>::exponent(code);
  return code != CODE_ONE ? stream_sum_squares<T, true, EMU, TAIL_SKIP, LANE>(xr, n, lane, cf, E)
                          : stream_sum_squares<T, false, EMU, TAIL_SKIP, LANE>(xr, n, lane, cf, E);
}

// Pass 3: x^ = h x~.
template <typename T, bool EMU, int OUTK = F64_EMU_OUTPUTS_OF_8>
__device__ __forceinline__ void stream_pass3(const T* __restrict__ xr, T* yr, int n, int lane, T h, int code) {
  const T cf = factor_of<T, true>(code);
  const int E = Pow2Scale<T>::exponent(code);
  if (code != CODE_ONE) stream_write<T, true, EMU, OUTK>(xr, yr, n, lane, h, cf, E);
  else stream_write<T, false, EMU, OUTK>(xr, yr, n, lane, h, cf, E);
}

// The hardware-operation passes of a binary64 vector that the integer-pipe
// steps do not take (rare: components 2^511 times smaller than the largest,
// subnormals with sigma_min, infinities, NaN).  Out of line, so that the
// common path of the kernels stays small in the instruction cache.
template <typename T, bool LANE = false>
__device__ __noinline__ T stream_pass2_slow(const T* __restrict__ xr, int n, int lane, int code) {
  return stream_pass2<T, false, true, LANE>(xr, n, lane, code);
}
template <typename T>
__device__ __noinline__ void stream_pass3_slow(const T* __restrict__ xr, T* yr, int n, int lane, T h, int code) {
  stream_pass3<T, false>(xr, yr, n, lane, h, code);
}

// Pass 2 and pass 3 of either kind: binary32 always uses the hardware
// operations inline; binary64 the integer-pipe steps inline when `emu`, the
// out-of-line hardware passes otherwise.
// TAIL_SKIP: the last, partial round adds only the chunks that hold terms
// (warp-uniform branches: a gain for short vectors; for the dense binary64
// rows, which have no partial round, the branches cost 6 % and are left out).
template <typename T, bool TAIL_SKIP = true, bool LANE = false>
__device__ __forceinline__ T stream_pass2_any(const T* __restrict__ xr, int n, int lane, int code, bool emu) {
  if (sizeof(T) == 4) return stream_pass2<T, false, TAIL_SKIP, LANE>(xr, n, lane, code);
  return emu ? stream_pass2<T, true, TAIL_SKIP, LANE>(xr, n, lane, code) : stream_pass2_slow<T, LANE>(xr, n, lane, code);
}
template <typename T, int OUTK = F64_EMU_OUTPUTS_OF_8>
__device__ __forceinline__ void stream_pass3_any(const T* __restrict__ xr, T* yr, int n, int lane, T h, int code,
                                                 bool emu) {
  if (sizeof(T) == 4) stream_pass3<T, false>(xr, yr, n, lane, h, code);
  else if (emu) stream_pass3<T, true, OUTK>(xr, yr, n, lane, h, code);
  else stream_pass3_slow<T>(xr, yr, n, lane, h, code);
}

// Passes 2 and 3 with the hardware operations, for any vector.
template <typename T>
__device__ __forceinline__ void warp_forward_stream_finish(const T* __restrict__ xr, T* yr, int n, int lane,
                                                           const VecOut<T>& out, int64_t vec, int code) {
  const T rt = FP<T>::sqrt(stream_pass2_any<T>(xr, n, lane, code, false));
  const T h = FP<T>::rcp(rt);
  if (yr) stream_pass3_any<T>(xr, yr, n, lane, h, code, false);
  if (lane == 0) out.put(vec, FP<T>::mul(inverse_of<T, true>(code), rt), h, code);
}

// No work between the passes (warp_forward_stream's default hook).
struct NoHook {
  __device__ __forceinline__ void operator()() const {}
};

// Forward, one warp per vector of any length (5 <= n <= 2^20), three passes
// over the vector: (1) largest magnitude and zero test, (2) scaled squares,
// (3) outputs.  yr may be null (norm only).  after_pass1() runs once pass 1
// has read the vector (a caller's prefetch of its next item).
template <typename T, typename Hook = NoHook>
__device__ __forceinline__ void warp_forward_stream(const T* __restrict__ xr, T* yr, int n, int lane,
                                                    const VecOut<T>& out, int64_t vec,
                                                    const Hook& after_pass1 = Hook()) {
  bool emu, have_s;
  T s;
  const int code = stream_pass1<T>(xr, yr, n, lane, out, vec, emu, s, have_s);
  after_pass1();
  if (code == CODE_ZERO) return;
  if (!have_s) s = stream_pass2_any<T>(xr, n, lane, code, emu);
  const T rt = FP<T>::sqrt(s);
  const T h = FP<T>::rcp(rt);
  if (yr) stream_pass3_any<T>(xr, yr, n, lane, h, code, emu);
  if (lane == 0) out.put(vec, FP<T>::mul(inverse_of<T, true>(code), rt), h, code);
}

// Forward of nb <= NB vectors by one warp, streaming: passes 1 and 2 of every
// vector, then one square root, one reciprocal and one norm product for the
// whole batch (lane j holds vector j's sum of squares), then pass 3 of every
// vector.  The binary64 square root and reciprocal take some twenty FP64
// instructions that the whole warp issues for one value; the batch shares
// them.  Same operations per vector as warp_forward_stream.  item(j, xr, yr,
// n, vec) describes vector j; it is called again in the third phase rather
// than keeping NB descriptors in registers.  Vectors longer than MAX_N are
// done one by one on the spot: between passes 2 and 3 the batch's vectors
// must stay in L1.  The loops over the batch are not unrolled: one copy of
// each pass keeps the kernel small.
// TAIL_SKIP as in stream_pass2_any: true for ragged vectors (partial last
// rounds), false for dense rows.
// OUTK: outputs of every 8 formed on the integer pipe (binary64).
template <typename T, int NB, int MAX_N, bool TAIL_SKIP = false, int OUTK = F64_EMU_OUTPUTS_OF_8, typename Item>
__device__ __forceinline__ void warp_forward_stream_batch(const Item& item, int nb, int lane, const VecOut<T>& out) {
  // binary64 batches of 2 or 4: the shuffle levels of all trees at once
  // (stream_tree_shfl2 / stream_tree_shfl4; binary64 forms no speculative
  // sums, so every sum comes from pass 2)
  constexpr bool PACK = (NB == 2 || NB == 4) && sizeof(T) == 8;
  T s = T(1);
  int code_l = CODE_ONE;  // lane j < nb: the code of vector j
  unsigned codes = 0;     // 2 bits per vector
  unsigned emu_m = 0;
  T part0 = T(0), part1 = T(0), part2 = T(0), part3 = T(0);  // PACK: lane partials of the vectors
  int len0 = 0, len1 = 0, len2 = 0, len3 = 0;
#pragma unroll 1
  for (int j = 0; j < NB; ++j) {
    int code = CODE_ZERO;
    if (j < nb) {
      const T* xr;
      T* yr;
      int n;
      int64_t vec;
      item(j, xr, yr, n, vec);
      bool emu, have_s;
      T sj;
      if (MAX_N < MAX_LEN && n > MAX_N) {
        warp_forward_stream<T>(xr, yr, n, lane, out, vec);
        code = CODE_ZERO;  // done
        emu = false;
      } else {
        code = stream_pass1<T>(xr, yr, n, lane, out, vec, emu, sj, have_s);
      }
      if (code != CODE_ZERO) {
        if (PACK) {
          const T pj = stream_pass2_any<T, TAIL_SKIP, true>(xr, n, lane, code, emu);
          if (j == 0) {
            part0 = pj;
            len0 = n;
          } else if (NB == 2 || j == 1) {  // (pairs: no registers for vectors 2 and 3)
            part1 = pj;
            len1 = n;
          } else if (j == 2) {
            part2 = pj;
            len2 = n;
          } else {
            part3 = pj;
            len3 = n;
          }
        } else {
          if (!have_s) sj = stream_pass2_any<T, TAIL_SKIP>(xr, n, lane, code, emu);
          if (lane == j) s = sj;
        }
        if (lane == j) code_l = code;
        emu_m |= (emu ? 1u : 0u) << j;
      }
    }
    codes |= (unsigned)code << (2 * j);
  }
  if (PACK && NB == 2) {
    const T r = stream_tree_shfl2<T>(part0, len0, part1, len1, lane);
    const T t0 = __shfl_sync(FULL, r, 0), t1 = __shfl_sync(FULL, r, 16);
    if (lane == 0 && (codes & 3u) != (unsigned)CODE_ZERO) s = t0;
    if (lane == 1 && ((codes >> 2) & 3u) != (unsigned)CODE_ZERO) s = t1;
  } else if (PACK) {
    const T r = stream_tree_shfl4<T>(part0, len0, part1, len1, part2, len2, part3, len3, lane);
    // totals: vector 0 in lane 0, 1 in lane 16, 2 in lane 8, 3 in lane 24
    const int src = lane < 4 ? ((lane & 1) << 4) | ((lane & 2) << 2) : 0;
    const T t = __shfl_sync(FULL, r, src);
    if (lane < 4 && ((codes >> (2 * lane)) & 3u) != (unsigned)CODE_ZERO) s = t;
  }
  const T rt = FP<T>::sqrt(s);
  const T h = FP<T>::rcp(rt);
  const T r = FP<T>::mul(inverse_of<T, true>(code_l), rt);
#pragma unroll 1
  for (int j = 0; j < NB; ++j) {
    const int code = (int)((codes >> (2 * j)) & 3u);
    if (code != CODE_ZERO) {
      const T* xr;
      T* yr;
      int n;
      int64_t vec;
      item(j, xr, yr, n, vec);
      const T hj = __shfl_sync(FULL, h, j);
      if (yr) stream_pass3_any<T, OUTK>(xr, yr, n, lane, hj, code, (emu_m >> j) & 1u);
      if (lane == j) out.put(vec, r, h, code);
    }
  }
}

// Steps 2-4 of the register-path forward: x~ = c x, the sum of squares in
// the order CR(n), r~ = sqrt, h = 1/r~, x^ = h x~, r = sigma r~.
template <typename T, int V, int CH, bool EMU>
__device__ __forceinline__ void warp_forward_tail(T (&v)[CH][V], T* yr, int n, int lane, const VecOut<T>& out,
                                                  int64_t vec, int code) {
  const T cf = factor_of<T, true>(code);
  T q[CH][V];
  {
    T (&vf)[CH * V] = reinterpret_cast<T (&)[CH * V]>(v);
    if (code != CODE_ONE) Chunk<T, CH * V, EMU>::scale(cf, Pow2Scale<T>::exponent(code), vf);  // warp-uniform
    Chunk<T, CH * V, EMU>::squares(vf, reinterpret_cast<T (&)[CH * V]>(q));
  }
  const T rt = FP<T>::sqrt(warp_cr_tree<T, V, CH>(q, n, lane));
  const T h = FP<T>::rcp(rt);
  if (yr) {
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      const int k0 = 32 * V * c + V * lane;
      if (k0 < n) {
        T o[V];
#pragma unroll
        for (int e = 0; e < V; ++e) o[e] = Chunk<T, CH * V, EMU>::template output<>(c * V + e, h, v[c][e]);
        Vec<T, V>::store(yr + k0, o);
      }
    }
  }
  if (lane == 0) out.put(vec, FP<T>::mul(inverse_of<T, true>(code), rt), h, code);
}

// Forward, one warp per vector of length 5 <= n <= 32 V CH (warp_forward).
// yr may be null (norm only).  The whole warp must call it with the same
// arguments.  warp_load reads the vector into registers, zero-padded.
template <typename T, int V, int CH>
__device__ __forceinline__ void warp_load(const T* __restrict__ xr, int n, int lane, T (&v)[CH][V]) {
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const int k0 = 32 * V * c + V * lane;
    if (k0 < n) {
      Vec<T, V>::load(xr + k0, v[c]);
    } else {
#pragma unroll
      for (int e = 0; e < V; ++e) v[c][e] = T(0);
    }
  }
}

// The same, on a row already in registers (warp_load), so that a kernel can
// have several rows' loads in flight before it computes.
template <typename T, int V, int CH>
__device__ __forceinline__ void warp_forward_loaded(T (&v)[CH][V], const T* __restrict__ xr, T* yr, int n, int lane,
                                                    const VecOut<T>& out, int64_t vec) {
  MagTrack<T> mt;
#pragma unroll
  for (int c = 0; c < CH; ++c) {
#pragma unroll
    for (int e = 0; e < V; ++e) mt.take(v[c][e]);  // zero padding changes neither m nor the zero test
  }
  mt.warp_reduce();
  if (mt.zero()) {  // every component compares equal to zero
    if (yr) {
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        const int k0 = 32 * V * c + V * lane;
        T z[V];
#pragma unroll
        for (int e = 0; e < V; ++e) z[e] = T(0);
        if (k0 < n) Vec<T, V>::store(yr + k0, z);
      }
    }
    if (lane == 0) out.put(vec, T(0), T(0), CODE_ZERO);
    return;
  }
  if (mt.has_nan()) {
    mt = MagTrack<T>();
#pragma unroll
    for (int c = 0; c < CH; ++c) {
#pragma unroll
      for (int e = 0; e < V; ++e) mt.take_skip_nan(v[c][e]);
    }
    mt.warp_reduce();
  }
  const int code = mt.code();
  if (sizeof(T) == 8 && !mt.emu_ok(code)) {
    // A binary64 vector with a component outside the range of the integer-pipe
    // steps: the streaming passes (loops, so the compiler cannot turn this
    // branch into predicated FP64 instructions on the common path) read it
    // again from cache.  Same order CR(n), same results.
    warp_forward_stream_finish<T>(xr, yr, n, lane, out, vec, code);
    return;
  }
  warp_forward_tail<T, V, CH, sizeof(T) == 8>(v, yr, n, lane, out, vec, code);
}

template <typename T, int V, int CH>
__device__ __forceinline__ void warp_forward(const T* __restrict__ xr, T* yr, int n, int lane,
                                             const VecOut<T>& out, int64_t vec) {
  T v[CH][V];
  warp_load<T, V, CH>(xr, n, lane, v);
  warp_forward_loaded<T, V, CH>(v, xr, yr, n, lane, out, vec);
}

// Backward pass 1 (dot = CR(y_k g_k)), streaming.  EMU (binary64): the
// products by f64emu::mul_signed, while `ry`, `rg` collect the integer keys of
// y and g that decide afterwards whether every product was in its range.
template <typename T, bool EMU>
__device__ __forceinline__ T bwd_dot_pass(const T* __restrict__ yr, const T* __restrict__ gr, int n, int lane,
                                          MagTrack<T>* ry, MagTrack<T>* rg) {
  T acc[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) acc[i] = T(0);
  for (int base = 0; base < n; base += 256) {
    T a[8], b[8];
    stream_load8(yr, base, n, lane, a);
    stream_load8(gr, base, n, lane, b);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if (base + 32 * i >= n) break;  // warp-uniform: no work for chunks past the end (acc[i] stays +0, unread)
      T q;
      if constexpr (EMU) {
        ry->take(a[i]);
        rg->take(b[i]);
        q = __longlong_as_double(static_cast<long long>(f64emu::mul_signed(
            static_cast<uint64_t>(__double_as_longlong(a[i])), static_cast<uint64_t>(__double_as_longlong(b[i])))));
      } else {
        q = FP<T>::mul(a[i], b[i]);
      }
      if (base == 0) acc[i] = q;
      else if (base + 32 * i + lane < n) acc[i] = FP<T>::add(acc[i], q);
    }
  }
  return stream_tree<T>(acc, n, lane);
}

template <typename T>
__device__ __noinline__ T bwd_dot_pass_slow(const T* __restrict__ yr, const T* __restrict__ gr, int n, int lane) {
  return bwd_dot_pass<T, false>(yr, gr, n, lane, nullptr, nullptr);
}

// Of every 8 products d_k h of the binary64 backward (d_k = g_k - y_k dot)
// on the integer-pipe path, how many are formed by f64emu::mul (the rest by
// the FP64 pipe), as F64_EMU_OUTPUTS_OF_8 for the forward's outputs.
// Measured on the ragged binary64 forward + backward workload (warp items):
// 0 / 1 / 2 / 3 / 4 / 8 of 8: 1.609 / 1.593 / 1.580 / 1.570 / 1.561 / 1.582 ms;
// with the group backward too (group_backward, chunks c < K): 3 / 4 / 5 / 6:
// 1.563 / 1.553 / 1.550 / 1.555 ms (1.568 at 4 without the groups).
constexpr int F64_EMU_GRAD_H_OF_8 = 4;
// Of every 8 differences d_k = RN(g_k - p_k) of that path, how many are
// formed by f64emu::add_signed (the upper chunks, i mod 8 >= 8 - K).
// Measured on the same workload (with the products by h at 4 of 8):
// 0 / 2 / 4 / 6 of 8: 1.553 / 1.595 / 1.690 / 1.853 ms -- the signed sum's
// alignment, normalization and rounding load the ALU more than the DADD it
// replaces loads the FP64 pipe, so none is taken.
constexpr int F64_EMU_GRAD_SUB_OF_8 = 0;

// Backward pass 2: grad_k = ((g_k - y_k dot) h) c.  SCALED = false skips the
// multiplication by c = 1 (exact, so the same bits).  EMU: y_k dot by
// f64emu::mul_signed.  HEMU (with EMU): F64_EMU_GRAD_H_OF_8 of every 8
// products d_k h by f64emu::mul and F64_EMU_GRAD_SUB_OF_8 of every 8
// differences by f64emu::add_signed (grad_h_in_range holds for the vector).
template <typename T, bool SCALED, bool EMU, bool HEMU = false>
__device__ __forceinline__ void bwd_grad_pass(const T* __restrict__ yr, const T* __restrict__ gr, T* gradr, int n,
                                              int lane, T dot, T h, T cf) {
  for (int base = 0; base < n; base += 256) {
    T a[8], b[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int k = base + 32 * i + lane;
      a[i] = k < n ? __ldcs(yr + k) : T(0);
      b[i] = k < n ? __ldcs(gr + k) : T(0);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if (base + 32 * i >= n) break;  // warp-uniform: no work for chunks past the end
      const int k = base + 32 * i + lane;
      T p;
      if constexpr (EMU)
        p = __longlong_as_double(static_cast<long long>(f64emu::mul_signed(
            static_cast<uint64_t>(__double_as_longlong(a[i])), static_cast<uint64_t>(__double_as_longlong(dot)))));
      else
        p = FP<T>::mul(a[i], dot);
      T d;
      if (HEMU && (i & 7) >= 8 - F64_EMU_GRAD_SUB_OF_8)  // compile-time per chunk
        d = __longlong_as_double(static_cast<long long>(
            f64emu::add_signed(static_cast<uint64_t>(__double_as_longlong(b[i])),
                               static_cast<uint64_t>(__double_as_longlong(p)) ^ 0x8000000000000000ull)));
      else
        d = FP<T>::sub(b[i], p);
      T o;
      if (HEMU && (i & 7) < F64_EMU_GRAD_H_OF_8)  // compile-time per chunk
        o = __longlong_as_double(static_cast<long long>(
            f64emu::mul(static_cast<uint64_t>(__double_as_longlong(d)), static_cast<uint64_t>(__double_as_longlong(h)))));
      else
        o = FP<T>::mul(d, h);
      if (SCALED) o = FP<T>::mul(o, cf);
      if (k < n) __stcs(gradr + k, o);
    }
  }
}

// Whether f64emu::mul_signed takes every product a_k b_k, from the keys of
// the a_k and of the b_k (MagTrack<double>: largest key, smallest nonzero
// key): true when either side is all zero, or both are finite and normal
// with 1 <= e_a + e_b - 1023 and e_a + e_b - 1023 <= 2045 for the extreme
// biased exponents.
__device__ __forceinline__ bool products_in_range(const MagTrack<double>& ta, const MagTrack<double>& tb) {
  if (ta.k == 0u || tb.k == 0u) return true;
  const uint32_t na = ta.kmin1 + 1u, nb = tb.kmin1 + 1u;  // smallest nonzero keys
  if (ta.k >= MagTrack<double>::HI_INF || tb.k >= MagTrack<double>::HI_INF) return false;
  if (na < (1u << 20) || nb < (1u << 20)) return false;  // a subnormal operand
  const int emin = (int)(na >> 20) + (int)(nb >> 20) - 1023, emax = (int)(ta.k >> 20) + (int)(tb.k >> 20) - 1023;
  return emin >= 1 && emax <= 2045;
}

// Whether f64emu::mul takes every product d_k h of the backward, with
// d_k = RN(g_k - p_k), p_k = RN(y_k dot), given the integer keys of y (ry),
// g (rg) and dot (rd), with products_in_range(ry, rd) already true (every p_k
// is zero or normal), and h > 0.  Biased exponents: a nonzero p_k lies in
// [e_y,lo + e_dot - 1023, e_y,hi + e_dot - 1021]; a nonzero difference of
// two values that are zero or normal with exponents >= E is a multiple of
// 2^(E - 1075), so its exponent is >= E - 52; and |g_k| + |p_k| is at most
// twice the largest value of exponent e_hi, which is the largest value of
// exponent e_hi + 1, so RN(g_k - p_k) stays at or below exponent e_hi + 1.
// mul() then needs d_k normal and e_d + e_h - 1023 within [1, 2045].
__device__ __forceinline__ bool grad_h_in_range(const MagTrack<double>& ry, const MagTrack<double>& rg,
                                                const MagTrack<double>& rd, double h) {
  const uint32_t hb = (uint32_t)((unsigned long long)__double_as_longlong(h) >> 32);
  const int eh = (int)(hb >> 20);  // the sign bit is part of eh: a negative h fails below
  if (eh < 1 || eh > 2046) return false;
  if (rg.k >= MagTrack<double>::HI_INF) return false;
  int elo = 4096, ehi = 0;
  if (rg.k != 0u) {
    const uint32_t ng = rg.kmin1 + 1u;  // smallest nonzero key of g
    if (ng < (1u << 20)) return false;  // a subnormal g_k
    elo = (int)(ng >> 20);
    ehi = (int)(rg.k >> 20);
  }
  if (ry.k != 0u && rd.k != 0u) {
    const int ed = (int)(rd.k >> 20);
    elo = min(elo, (int)((ry.kmin1 + 1u) >> 20) + ed - 1023);
    ehi = max(ehi, (int)(ry.k >> 20) + ed - 1021);
  }
  if (ehi == 0) return true;  // every d_k is zero
  const int dlo = elo - 52, dhi = ehi + 1;
  // ehi <= 2045 also lets f64emu::add_signed form every d_k (no overflow)
  return ehi <= 2045 && dlo >= 1 && dlo + eh - 1023 >= 1 && dhi + eh - 1023 <= 2045;
}

// Backward, one warp per vector of any length: (1) dot = CR(y_k g_k),
// (2) grad_k = ((g_k - y_k dot) h) c.  binary64 forms the products on the
// integer pipes when every one of them is in range (pass 1 runs that way
// speculatively and runs again with the hardware products otherwise).
template <typename T>
__device__ __forceinline__ void warp_backward_stream(const T* __restrict__ yr, const T* __restrict__ gr, T* gradr,
                                                     int n, int lane, T h, int code) {
  if (code == CODE_ZERO) {
    for (int k = lane; k < n; k += 32) __stcs(gradr + k, T(0));
    return;
  }
  const T cf = factor_of<T, true>(code);
  if constexpr (sizeof(T) == 8) {
    MagTrack<T> ry, rg;
    T dot = bwd_dot_pass<T, true>(yr, gr, n, lane, &ry, &rg);
    ry.warp_reduce();
    rg.warp_reduce();
    if (!products_in_range(ry, rg)) dot = bwd_dot_pass_slow<T>(yr, gr, n, lane);
    MagTrack<T> rd;
    rd.take(dot);
    const bool emu = products_in_range(ry, rd);
    if (emu && F64_EMU_GRAD_H_OF_8 > 0 && grad_h_in_range(ry, rg, rd, h)) {
      if (code != CODE_ONE) bwd_grad_pass<T, true, true, true>(yr, gr, gradr, n, lane, dot, h, cf);
      else bwd_grad_pass<T, false, true, true>(yr, gr, gradr, n, lane, dot, h, cf);
    } else if (emu) {
      if (code != CODE_ONE) bwd_grad_pass<T, true, true>(yr, gr, gradr, n, lane, dot, h, cf);
      else bwd_grad_pass<T, false, true>(yr, gr, gradr, n, lane, dot, h, cf);
    } else {
      if (code != CODE_ONE) bwd_grad_pass<T, true, false>(yr, gr, gradr, n, lane, dot, h, cf);
      else bwd_grad_pass<T, false, false>(yr, gr, gradr, n, lane, dot, h, cf);
    }
  } else {
    const T dot = bwd_dot_pass<T, false>(yr, gr, n, lane, nullptr, nullptr);
    if (code != CODE_ONE) bwd_grad_pass<T, true, false>(yr, gr, gradr, n, lane, dot, h, cf);
    else bwd_grad_pass<T, false, false>(yr, gr, gradr, n, lane, dot, h, cf);
  }
}

}  // namespace ngb
