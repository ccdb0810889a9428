// ngb_arith.cuh -- device arithmetic of the scaling normalization of
// Mascarenhas, "Fast and accurate normalization of vectors and quaternions"
// (arXiv 1606.06508), as inline device functions shared by every kernel.
//
// Every floating-point step is one correctly rounded IEEE operation through
// the __*_rn intrinsics (round to nearest even, never contracted into a fused
// multiply-add), and the library is built with -ftz=false -prec-div=true
// -prec-sqrt=true -fmad=false: the error analysis of the paper assumes IEEE
// arithmetic with gradual underflow (Section 3, remark on DAZ/FTZ).  The
// operations run in the order of Algorithms 3-7 so that results are
// bit-identical to a sequential evaluation of the same steps.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "ngb_f64emu.cuh"

namespace ngb {

enum : int { CODE_ONE = 0, CODE_SIGMA_MIN = 1, CODE_SIGMA_MAX = 2, CODE_ZERO = 3 };

// Canonical summation order for n >= 5: CR_SLOTS slots, slot j holding the
// left-to-right sum of terms j, j + CR_SLOTS, ...; then a halving tree over
// the slots with strides CR_SLOTS/2 .. 1, skipping slots that hold no term.
// 256 slots: a warp streams any length with 8 partial sums per lane, and a
// block of 256 threads holds one slot per thread.
constexpr int CR_SLOTS = 256;
constexpr int MAX_LEN = 1 << 20;

template <typename T> struct FP;

template <> struct FP<float> {
  __device__ __forceinline__ static float mul(float a, float b) { return __fmul_rn(a, b); }
  __device__ __forceinline__ static float add(float a, float b) { return __fadd_rn(a, b); }
  __device__ __forceinline__ static float sub(float a, float b) { return __fsub_rn(a, b); }
  __device__ __forceinline__ static float div(float a, float b) { return __fdiv_rn(a, b); }
  __device__ __forceinline__ static float sqrt(float a) { return __fsqrt_rn(a); }
  __device__ __forceinline__ static float rcp(float a) { return __frcp_rn(a); }
  __device__ __forceinline__ static float abs(float a) { return fabsf(a); }
  __device__ __forceinline__ static float fmax(float a, float b) { return fmaxf(a, b); }
  // Table 2, binary32 row (n <= 4)
  static constexpr float tau_min = 0x1p-49f, sigma_min = 0x1p100f, inv_sigma_min = 0x1p-100f;
  static constexpr float tau_max = 0x1p62f, sigma_max = 0x1p-66f, inv_sigma_max = 0x1p66f;
  // 5 <= n <= 2^20: tau_max = 2^floor((log2(omega) - 21) / 2), sigma_max * omega <= tau_max
  static constexpr float tau_max_n = 0x1p53f, sigma_max_n = 0x1p-75f, inv_sigma_max_n = 0x1p75f;
};

template <> struct FP<double> {
  __device__ __forceinline__ static double mul(double a, double b) { return __dmul_rn(a, b); }
  __device__ __forceinline__ static double add(double a, double b) { return __dadd_rn(a, b); }
  __device__ __forceinline__ static double sub(double a, double b) { return __dsub_rn(a, b); }
  __device__ __forceinline__ static double div(double a, double b) { return __ddiv_rn(a, b); }
  __device__ __forceinline__ static double sqrt(double a) { return __dsqrt_rn(a); }
  __device__ __forceinline__ static double rcp(double a) { return __drcp_rn(a); }
  __device__ __forceinline__ static double abs(double a) { return fabs(a); }
  __device__ __forceinline__ static double fmax(double a, double b) { return ::fmax(a, b); }
  // Table 2, binary64 row (n <= 4)
  static constexpr double tau_min = 0x1p-482, sigma_min = 0x1p592, inv_sigma_min = 0x1p-592;
  static constexpr double tau_max = 0x1p510, sigma_max = 0x1p-514, inv_sigma_max = 0x1p514;
  static constexpr double tau_max_n = 0x1p501, sigma_max_n = 0x1p-523, inv_sigma_max_n = 0x1p523;
  static constexpr int tau_min_exp = -482, tau_max_n_exp = 501;  // log2 of tau_min, tau_max_n
  static constexpr int tau_max_exp = 510, sigma_min_exp = 592, sigma_max_exp = -514;  // log2, n <= 4
};

// The factor choice of Scale2D/Scale3D/Normalize4D: compare the largest
// magnitude m with tau_min and tau_max.  A NaN m fails both comparisons and
// takes the sigma_min branch, as in the paper.
template <typename T, bool GENERIC>
__device__ __forceinline__ int select_code(T m) {
  const T tmax = GENERIC ? FP<T>::tau_max_n : FP<T>::tau_max;
  if (m >= FP<T>::tau_min) {
    if (m <= tmax) return CODE_ONE;
    return CODE_SIGMA_MAX;
  }
  return CODE_SIGMA_MIN;
}

// c, the factor applied to x (x~ = c x)
template <typename T, bool GENERIC>
__device__ __forceinline__ T factor_of(int code) {
  const T smax = GENERIC ? FP<T>::sigma_max_n : FP<T>::sigma_max;
  return code == CODE_SIGMA_MIN ? FP<T>::sigma_min : (code == CODE_SIGMA_MAX ? smax : T(1));
}

// sigma = 1/c, the first value returned by Scale2D/Scale3D (r^ = sigma r~)
template <typename T, bool GENERIC>
__device__ __forceinline__ T inverse_of(int code) {
  const T ismax = GENERIC ? FP<T>::inv_sigma_max_n : FP<T>::inv_sigma_max;
  return code == CODE_SIGMA_MIN ? FP<T>::inv_sigma_min : (code == CODE_SIGMA_MAX ? ismax : T(1));
}

// x~ = c x; with c = 1 the input is used as it is (as the algorithms return x).
template <typename T>
__device__ __forceinline__ T scale_by(int code, T c, T x) {
  return code == CODE_ONE ? x : FP<T>::mul(c, x);
}

// Largest magnitude of a vector of n >= 5 components, for the factor choice
// with the generic constants, and the zero test.  It only has to decide
// m >= tau_min, m <= tau_max and "every component is zero", with m the
// largest |x_k| over the components that are not NaN.
//   binary32: m = fmax over |x_k| (fmax skips a NaN operand) and a nonzero flag.
//   binary64: integer keys, so that no FP64 instruction runs per component.
//     key(x) = (high word of |x|) | (low word != 0), maxed as unsigned.  tau_min
//     and tau_max are powers of two: low word zero, even high word h(tau).
//     Then |x| >= tau <=> key >= h(tau) and |x| > tau <=> key > h(tau), so the
//     largest key decides both comparisons for m; the vector is zero iff the
//     largest key is 0; and a NaN component (key > h(+inf)) is detected, after
//     which the caller takes the keys again with NaN components counted as 0.
template <typename T> struct MagTrack;

template <> struct MagTrack<float> {
  float m = 0.0f;
  bool nz = false;
  __device__ __forceinline__ void take(float v) {
    nz |= !(v == 0.0f);
    m = fmaxf(m, fabsf(v));
  }
  __device__ __forceinline__ void take_skip_nan(float v) { take(v); }
  __device__ __forceinline__ void merge(const MagTrack& o) {
    nz |= o.nz;
    m = fmaxf(m, o.m);
  }
  __device__ __forceinline__ void warp_reduce() {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    nz = __any_sync(0xffffffffu, nz);
  }
  __device__ __forceinline__ bool zero() const { return !nz; }
  __device__ __forceinline__ bool has_nan() const { return false; }
  __device__ __forceinline__ int code() const { return select_code<float, true>(m); }
  __device__ __forceinline__ bool emu_ok(int /*code*/) const { return false; }
};

template <> struct MagTrack<double> {
  static constexpr uint32_t HI_INF = 0x7FF00000u;
  static constexpr uint32_t HI_TMIN = (uint32_t)(FP<double>::tau_min_exp + 1023) << 20;
  static constexpr uint32_t HI_TMAX = (uint32_t)(FP<double>::tau_max_n_exp + 1023) << 20;
  uint32_t k = 0;
  uint32_t kmin1 = 0xFFFFFFFFu;  // min over components of key - 1: zero components wrap to the top
  __device__ __forceinline__ static uint32_t key(double v) {
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(v));
    const uint32_t lo = (uint32_t)b;
    return ((uint32_t)(b >> 32) & 0x7FFFFFFFu) | (lo < 1u ? lo : 1u);
  }
  __device__ __forceinline__ void take(double v) {
    const uint32_t t = key(v);
    k = max(k, t);
    kmin1 = min(kmin1, t - 1u);
  }
  __device__ __forceinline__ void take_skip_nan(double v) {  // also rules out the integer-pipe steps
    const uint32_t t = key(v);
    k = max(k, t > HI_INF ? 0u : t);
    kmin1 = 0u;
  }
  __device__ __forceinline__ void merge(const MagTrack& o) {
    k = max(k, o.k);
    kmin1 = min(kmin1, o.kmin1);
  }
  __device__ __forceinline__ void warp_reduce() {
    k = __reduce_max_sync(0xffffffffu, k);
    kmin1 = __reduce_min_sync(0xffffffffu, kmin1);
  }
  __device__ __forceinline__ bool zero() const { return k == 0u; }
  __device__ __forceinline__ bool has_nan() const { return k > HI_INF; }
  __device__ __forceinline__ int code() const {
    if (k >= HI_TMIN) return k <= HI_TMAX ? CODE_ONE : CODE_SIGMA_MAX;
    return CODE_SIGMA_MIN;
  }
  // Whether the integer-pipe scale and squares (Chunk<double, N, true>) take
  // every component of the vector for the factor c = 2^E of `code`: no NaN or
  // infinity, and every nonzero component normal with 2^-511 <= |c x_k| <
  // 2^512.  The upper bound holds for every factor choice (|c x_k| <= 2^501
  // with c = 1, < 2^501 with sigma_max, < 2^110 with sigma_min); the lower
  // bound is |x_k| >= 2^(-511 - E), i.e. key >= (512 - E) << 20, and at least
  // the smallest normal number.
  __device__ __forceinline__ bool emu_ok(int code) const {
    const int E = code == CODE_ONE ? 0 : (code == CODE_SIGMA_MIN ? 592 : -523);
    const int p = 512 - E;
    const uint32_t tmin = p > 1 ? (uint32_t)p << 20 : (1u << 20);
    return k < HI_INF && kmin1 >= tmin - 1u;
  }
};

// x~ = c x for c = 2^E != 1 (generic constants).  binary64: when x and c x are
// both normal the product is exact and is formed by adding E to the exponent
// field, which gives the bits of RN(c x); zeros, subnormals, infinities, NaN
// and subnormal results take the multiplication.  binary32 multiplies.
template <typename T> struct Pow2Scale;
template <> struct Pow2Scale<float> {
  __device__ __forceinline__ static float apply(float c, int /*E*/, float x) { return __fmul_rn(c, x); }
  __device__ __forceinline__ static int exponent(int code) { return code == CODE_SIGMA_MIN ? 100 : -75; }
};
template <> struct Pow2Scale<double> {
  __device__ __forceinline__ static double apply(double c, int E, double x) {
    const long long b = __double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7ff);
    const int ne = e + E;
    if (e != 0 && e != 0x7ff && ne > 0 && ne < 0x7ff) return __longlong_as_double(b + ((long long)E << 52));
    return __dmul_rn(c, x);
  }
  __device__ __forceinline__ static int exponent(int code) { return code == CODE_SIGMA_MIN ? 592 : -523; }
};

// Chunk operations of the long-vector paths, N values per thread:
//   scale:   v_i <- c v_i with c = 2^E != 1 (exact in every case the paper
//            allows: the factor only moves the exponent)
//   squares: q_i <- RN(v_i * v_i)
// EMU = false: the hardware multiplication.  EMU = true (binary64 only): the
// integer-pipe forms, exponent addition for the scale and f64emu::square for
// the squares; the caller takes this form only for a vector whose components
// are all in their range (MagTrack<double>::emu_ok), so no component needs a
// fallback and no FP64 instruction is issued for these steps.
// Of every 8 outputs x^_k = h x~_k of a binary64 vector on the integer-pipe
// path, how many are formed by f64emu::mul (the rest by the FP64 pipe): the
// two pipes run side by side, and this split balances them.  Measured (0 to
// 8 of 8): ragged binary64 0.40 / 0.42 / 0.43 / 0.42 / 0.41 / 0.34 / 0.33 of
// the copy bandwidth at 0 / 1 / 2 / 3 / 4 / 6 / 8; dense rows 0.44 at 2 and 4.
// (The dense binary64 row batch takes 3: rows of 256, 2^19 rows, 0.739 ms at
// 2 and 0.712 ms at 3, while the ragged binary64 workloads are fastest at 2:
// forward 6.96 / 7.00 / 7.03 ms at 2 / 1 / 3.)
constexpr int F64_EMU_OUTPUTS_OF_8 = 2;

template <typename T, int N, bool EMU> struct Chunk {
  __device__ __forceinline__ static void scale(T c, int /*E*/, T (&v)[N]) {
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = FP<T>::mul(c, v[i]);
  }
  __device__ __forceinline__ static void squares(const T (&v)[N], T (&q)[N]) {
#pragma unroll
    for (int i = 0; i < N; ++i) q[i] = FP<T>::mul(v[i], v[i]);
  }
  template <int K = F64_EMU_OUTPUTS_OF_8>
  __device__ __forceinline__ static T output(int /*i*/, T h, T v) { return FP<T>::mul(h, v); }
};
template <int N> struct Chunk<double, N, true> {
  __device__ __forceinline__ static void scale(double /*c*/, int E, double (&v)[N]) {
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(v[i]));
      const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
      const bool zero = ((hi << 1) | lo) == 0u;  // c (+-0) = +-0
      const uint32_t nhi = zero ? hi : hi + ((uint32_t)E << 20);
      v[i] = __longlong_as_double(static_cast<long long>(((unsigned long long)nhi << 32) | lo));
    }
  }
  __device__ __forceinline__ static void squares(const double (&v)[N], double (&q)[N]) {
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const uint64_t a = static_cast<uint64_t>(__double_as_longlong(v[i])) & 0x7FFFFFFFFFFFFFFFull;
      q[i] = __longlong_as_double(static_cast<long long>(f64emu::square(a)));
    }
  }
  // x^ = RN(h x~) for chunk position i (h = 1/r~ lies in [2^-511, 2^482] and
  // h x~ in [2^-1022, 1] for these vectors, inside f64emu::mul's range)
  // (K of every 8 by f64emu::mul: F64_EMU_OUTPUTS_OF_8 unless a kernel asks otherwise)
  template <int K = F64_EMU_OUTPUTS_OF_8>
  __device__ __forceinline__ static double output(int i, double h, double v) {
    if ((i & 7) < K)
      return __longlong_as_double(static_cast<long long>(
          f64emu::mul(static_cast<uint64_t>(__double_as_longlong(v)), static_cast<uint64_t>(__double_as_longlong(h)))));
    return __dmul_rn(h, v);
  }
};

// ---------------------------------------------------------------------------
// The largest magnitude of n <= 4 components in the branch order of Scale2D
// (Algorithm 3), Scale3D (Algorithm 4) and Normalize4D (Algorithm 7).
// Returns true for the zero result.  Readings: in Normalize4D the assignment
// m <- |x4| belongs to an omitted Else; the zero result needs every component
// equal to zero (in the branches that reach "m = 0" the components that were
// not compared with ">=" may still be NaN, and a NaN input must give NaN).
template <typename T, int D> struct SmallMax;

template <typename T> struct SmallMax<T, 1> {
  __device__ __forceinline__ static bool run(const T* x, T& m) {
    m = FP<T>::abs(x[0]);
    return m == T(0);
  }
};

template <typename T> struct SmallMax<T, 2> {
  __device__ __forceinline__ static bool run(const T* x, T& m) {
    m = FP<T>::abs(x[0]);
    if (m >= FP<T>::abs(x[1])) {
      if (m == T(0)) return true;
    } else {
      m = FP<T>::abs(x[1]);
    }
    return false;
  }
};

template <typename T> struct SmallMax<T, 3> {
  __device__ __forceinline__ static bool run(const T* x, T& m) {
    m = FP<T>::abs(x[0]);
    if (m < FP<T>::abs(x[1])) {
      m = FP<T>::abs(x[1]);
      if (m < FP<T>::abs(x[2])) m = FP<T>::abs(x[2]);
    } else {
      if (m >= FP<T>::abs(x[2])) {
        if (m == T(0) && x[1] == T(0)) return true;
      } else {
        m = FP<T>::abs(x[2]);
      }
    }
    return false;
  }
};

template <typename T> struct SmallMax<T, 4> {
  __device__ __forceinline__ static bool run(const T* x, T& m) {
    m = FP<T>::abs(x[0]);
    if (m < FP<T>::abs(x[1])) {
      m = FP<T>::abs(x[1]);
      if (m < FP<T>::abs(x[2])) m = FP<T>::abs(x[2]);
      if (m < FP<T>::abs(x[3])) m = FP<T>::abs(x[3]);
    } else {
      if (m < FP<T>::abs(x[2])) {
        m = FP<T>::abs(x[2]);
        if (m < FP<T>::abs(x[3])) m = FP<T>::abs(x[3]);
      } else {
        if (m >= FP<T>::abs(x[3])) {
          if (m == T(0) && x[1] == T(0) && x[2] == T(0)) return true;
        } else {
          m = FP<T>::abs(x[3]);
        }
      }
    }
    return false;
  }
};

// Normalize2D / Normalize3D / Normalize4D (Algorithms 5-7; n = 1 runs the same
// steps on one component) with the hardware operations.  x and y may be the
// same array.  quat_zero picks the [0, 0, 1, 0] zero result of Algorithm 7
// for D = 4.  Returns the factor code; r = sigma r~, h = 1/r~.
template <typename T, int D>
__device__ __forceinline__ int normalize_small_hw(const T* x, T* y, T& r, T& h, bool quat_zero) {
  T m;
  if (SmallMax<T, D>::run(x, m)) {
#pragma unroll
    for (int k = 0; k < D; ++k) y[k] = T(0);
    if (D == 4 && quat_zero) y[2] = T(1);
    r = T(0);
    h = T(0);
    return CODE_ZERO;
  }
  const int code = select_code<T, false>(m);
  const T c = factor_of<T, false>(code);
  T t[D];
#pragma unroll
  for (int k = 0; k < D; ++k) t[k] = scale_by(code, c, x[k]);
  T s = FP<T>::mul(t[0], t[0]);
#pragma unroll
  for (int k = 1; k < D; ++k) s = FP<T>::add(s, FP<T>::mul(t[k], t[k]));
  const T rt = FP<T>::sqrt(s);
  h = FP<T>::rcp(rt);
  r = FP<T>::mul(inverse_of<T, false>(code), rt);
#pragma unroll
  for (int k = 0; k < D; ++k) y[k] = FP<T>::mul(h, t[k]);
  return code;
}

// binary64 vectors of n <= 4 on the integer pipes (Algorithms 5-7 with the
// operations of f64emu).  Components beyond n are zero: a zero changes
// neither the largest magnitude nor the sum (s + 0 = s), so one form serves
// every n <= D.
//
// The largest magnitude m and the zero test come from the integer keys of
// |x_k| (MagTrack<double>::key); tau_min and tau_max are powers of two, so
// the largest key decides m >= tau_min and m <= tau_max exactly, and for
// finite components the branch order of Scale2D/Scale3D/Normalize4D only
// reaches that same maximum.  The form is taken when every component is
// finite and every nonzero one is normal with |c x_k| >= 2^-511 (keys from
// (512 - E) << 20 up, c = 2^E); then, with the n <= 4 row of Table 2:
//   |c x_k| < 2^511 (c = 1: m <= 2^510; sigma_max: m 2^-514 < 2^510;
//     sigma_min: m 2^592 < 2^110), so every square is normal and below 2^1022
//     and s <= 4 2^1020 stays finite;
//   s >= (c m)^2 >= 2^-964 (c = 1: m >= 2^-482; sigma_min: m >= 2^-1022;
//     sigma_max: m > 2^510), so r~ = sqrt(s) lies in [2^-482, 2^511], 1/r~ is
//     normal, and h c x_k is 0 or normal (|h| >= 2^-511, |c x_k| >= 2^-511);
//   r^ = sigma r~ is a power-of-two scaling (f64emu::ldexp_rn: the overflow
//     to infinity and the subnormal rounding included).
// c x_k is an exponent addition (exact: x_k and c x_k are normal); the
// squares, the sum in the order of the algorithms, the square root and the
// reciprocal are f64emu's correctly rounded operations, and the outputs
// h c x_k the FP64 pipe's multiplication (SMALL_F64_FP64_OUTPUTS), which
// runs beside the integer work.  Vectors outside the range take
// normalize_small_hw.  Measured on 2^25 binary64 quaternions: 1.34 ms with
// every step on the integer pipes, 1.14 ms with the outputs on the FP64 pipe
// (3 and 2 components: -17 % and -14 %); the FP64 path alone needs about 95
// FP64 instructions per quaternion, about 6 ms.
constexpr bool SMALL_F64_INTEGER = true;
constexpr bool SMALL_F64_FP64_OUTPUTS = true;

template <int D>
struct SmallKeysF64 {
  int code;  // CODE_ZERO for the zero vector
  int E;     // c = 2^E
  bool ok;   // the integer-pipe form takes this vector
  __device__ __forceinline__ explicit SmallKeysF64(const double* x) {
    constexpr uint32_t HI_INF = 0x7FF00000u;
    constexpr uint32_t HI_TMIN = (uint32_t)(FP<double>::tau_min_exp + 1023) << 20;
    constexpr uint32_t HI_TMAX = (uint32_t)(FP<double>::tau_max_exp + 1023) << 20;
    uint32_t k = 0, kmin1 = 0xFFFFFFFFu;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const uint32_t t = MagTrack<double>::key(x[d]);
      k = max(k, t);
      kmin1 = min(kmin1, t - 1u);  // zero components wrap to the top
    }
    code = k >= HI_TMIN ? (k <= HI_TMAX ? CODE_ONE : CODE_SIGMA_MAX) : CODE_SIGMA_MIN;
    E = code == CODE_ONE ? 0 : (code == CODE_SIGMA_MIN ? FP<double>::sigma_min_exp : FP<double>::sigma_max_exp);
    const int p = 512 - E;
    const uint32_t tmin = p > 1 ? (uint32_t)p << 20 : (1u << 20);
    ok = k < HI_INF && kmin1 >= tmin - 1u;
    if (k == 0u) code = CODE_ZERO;
  }
};

// FP64_SQUARES: form the squares x~_k^2 with the FP64 pipe's multiplication
// instead of f64emu::square (the same bits: in this range every square is a
// normal number, and both are the correctly rounded product).  Measured on
// 2^25 binary64 quaternions whose components all lie in range: 0.85 ms
// against 0.98 ms with the integer squares; on the wide-exponent recipe,
// where many vectors take the hardware steps and already load the FP64 pipe,
// the FP64 squares were 7 % slower.  The dense kernels therefore choose them
// per warp, when every vector of the warp is in range (normalize_small_warp).
template <int D, bool FP64_SQUARES = false>
__device__ __forceinline__ int normalize_small_f64_int(const double* x, double* y, double& r, double& h,
                                                       bool quat_zero, const SmallKeysF64<D>& kk) {
  if (kk.code == CODE_ZERO) {
#pragma unroll
    for (int d = 0; d < D; ++d) y[d] = 0.0;
    if (D == 4 && quat_zero) y[2] = 1.0;
    r = 0.0;
    h = 0.0;
    return CODE_ZERO;
  }
  constexpr uint64_t ABS = 0x7FFFFFFFFFFFFFFFull;
  const uint64_t shift = (uint64_t)((int64_t)kk.E * (int64_t(1) << 52));
  uint64_t t[D];
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const uint64_t b = static_cast<uint64_t>(__double_as_longlong(x[d]));
    t[d] = (b << 1) == 0 ? b : b + shift;  // c (+-0) = +-0
  }
  auto square = [](uint64_t a) {
    if constexpr (FP64_SQUARES) {
      const double v = __longlong_as_double(static_cast<long long>(a));
      return static_cast<uint64_t>(__double_as_longlong(__dmul_rn(v, v)));
    }
    return f64emu::square(a);
  };
  bool finite;  // always true here: s < 2^1023
  uint64_t s = square(t[0] & ABS);
#pragma unroll
  for (int d = 1; d < D; ++d) s = f64emu::add_nonneg(s, square(t[d] & ABS), finite);
  const uint64_t rt = f64emu::sqrt_rn(s);
  const uint64_t hb = f64emu::rcp_rn(rt);
#pragma unroll
  for (int d = 0; d < D; ++d) {
    if (SMALL_F64_FP64_OUTPUTS)
      y[d] = __dmul_rn(__longlong_as_double(static_cast<long long>(hb)), __longlong_as_double(static_cast<long long>(t[d])));
    else
      y[d] = __longlong_as_double(static_cast<long long>(f64emu::mul(t[d], hb)));
  }
  r = __longlong_as_double(static_cast<long long>(f64emu::ldexp_rn(rt, -kk.E)));
  h = __longlong_as_double(static_cast<long long>(hb));
  return kk.code;
}

// Normalize2D / Normalize3D / Normalize4D: binary64 vectors in the range of
// the integer-pipe form take it, every other vector the hardware operations
// (both give the same bits).
template <typename T, int D>
__device__ __forceinline__ int normalize_small(const T* x, T* y, T& r, T& h, bool quat_zero) {
  if constexpr (sizeof(T) == 8 && SMALL_F64_INTEGER) {
    const SmallKeysF64<D> kk(x);
    if (kk.ok) return normalize_small_f64_int<D>(x, y, r, h, quat_zero, kk);
  }
  return normalize_small_hw<T, D>(x, y, r, h, quat_zero);
}

// normalize_small for one vector per lane, called by all 32 lanes of a warp
// together (lanes without a vector pass active = false and zero components,
// and get no result).  binary64: when every vector of the warp is in the
// range of the integer-pipe form, the squares go to the FP64 pipe
// (normalize_small_f64_int); otherwise in-range vectors keep the integer
// squares and the others take the hardware steps.  Same results either way.
template <typename T, int D>
__device__ __forceinline__ int normalize_small_warp(const T* x, T* y, T& r, T& h, bool quat_zero, bool active) {
  if constexpr (sizeof(T) == 8 && SMALL_F64_INTEGER) {
    const SmallKeysF64<D> kk(x);
    const bool all_in_range = __all_sync(0xffffffffu, kk.ok || !active);
    if (!active) return CODE_ZERO;
    if (!kk.ok) return normalize_small_hw<T, D>(x, y, r, h, quat_zero);
    // warp-uniform: one copy of the steps per choice, no per-square select
    if (all_in_range) return normalize_small_f64_int<D, true>(x, y, r, h, quat_zero, kk);
    return normalize_small_f64_int<D, false>(x, y, r, h, quat_zero, kk);
  } else {
    if (!active) return CODE_ZERO;
    return normalize_small<T, D>(x, y, r, h, quat_zero);
  }
}

// Backward of y = x/|x| for n <= 4: dot = y.g left to right,
// grad_k = ((g_k - y_k dot) h) c; zero input -> grad = +0.
template <typename T, int D>
__device__ __forceinline__ void backward_small(const T* y, const T* g, T h, int code, T* grad) {
  if (code == CODE_ZERO) {
#pragma unroll
    for (int k = 0; k < D; ++k) grad[k] = T(0);
    return;
  }
  const T c = factor_of<T, false>(code);
  T dot = FP<T>::mul(y[0], g[0]);
#pragma unroll
  for (int k = 1; k < D; ++k) dot = FP<T>::add(dot, FP<T>::mul(y[k], g[k]));
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const T tk = FP<T>::sub(g[k], FP<T>::mul(y[k], dot));
    grad[k] = FP<T>::mul(FP<T>::mul(tk, h), c);
  }
}

// ---------------------------------------------------------------------------
// One thread, 5 <= n <= NMAX (NMAX <= CR_SLOTS): the generic steps with the
// order CR(n), every slot holding one term.
template <typename T, int NMAX>
__device__ __forceinline__ T cr_sum_thread(T (&q)[NMAX], int n) {
#pragma unroll
  for (int s = NMAX / 2; s >= 1; s /= 2) {
#pragma unroll
    for (int j = 0; j < s; ++j)
      if (j + s < n) q[j] = FP<T>::add(q[j], q[j + s]);
  }
  return q[0];
}

template <typename T, int NMAX>
__device__ __forceinline__ int normalize_thread_generic(const T* __restrict__ xr, T* yr, int n, T& r, T& h) {
  T v[NMAX];
  MagTrack<T> mt;
#pragma unroll
  for (int k = 0; k < NMAX; ++k) {
    v[k] = k < n ? xr[k] : T(0);
    if (k < n) mt.take(v[k]);
  }
  if (mt.zero()) {
    if (yr)
      for (int k = 0; k < n; ++k) yr[k] = T(0);
    r = T(0);
    h = T(0);
    return CODE_ZERO;
  }
  if (mt.has_nan()) {
    mt = MagTrack<T>();
#pragma unroll
    for (int k = 0; k < NMAX; ++k)
      if (k < n) mt.take_skip_nan(v[k]);
  }
  const int code = mt.code();
  const T c = factor_of<T, true>(code);
  T q[NMAX];
#pragma unroll
  for (int k = 0; k < NMAX; ++k) {
    v[k] = scale_by(code, c, v[k]);
    q[k] = FP<T>::mul(v[k], v[k]);
  }
  const T rt = FP<T>::sqrt(cr_sum_thread<T, NMAX>(q, n));
  h = FP<T>::rcp(rt);
  r = FP<T>::mul(inverse_of<T, true>(code), rt);
  if (yr) {
#pragma unroll
    for (int k = 0; k < NMAX; ++k)
      if (k < n) yr[k] = FP<T>::mul(h, v[k]);
  }
  return code;
}

template <typename T, int NMAX>
__device__ __forceinline__ void backward_thread_generic(const T* __restrict__ yr, const T* __restrict__ gr, int n,
                                                        T h, int code, T* gradr) {
  if (code == CODE_ZERO) {
    for (int k = 0; k < n; ++k) gradr[k] = T(0);
    return;
  }
  const T c = factor_of<T, true>(code);
  T yv[NMAX], gv[NMAX], q[NMAX];
#pragma unroll
  for (int k = 0; k < NMAX; ++k) {
    yv[k] = k < n ? yr[k] : T(0);
    gv[k] = k < n ? gr[k] : T(0);
    q[k] = FP<T>::mul(yv[k], gv[k]);
  }
  const T dot = cr_sum_thread<T, NMAX>(q, n);
#pragma unroll
  for (int k = 0; k < NMAX; ++k)
    if (k < n) gradr[k] = FP<T>::mul(FP<T>::mul(FP<T>::sub(gv[k], FP<T>::mul(yv[k], dot)), h), c);
}

// Per-vector outputs (each pointer nullable).
template <typename T>
struct VecOut {
  T* norm;
  T* saved_h;
  int8_t* saved_code;
  __device__ __forceinline__ void put(int64_t i, T r, T h, int code) const {
    if (norm) norm[i] = r;
    if (saved_h) saved_h[i] = h;
    if (saved_code) saved_code[i] = (int8_t)code;
  }
};

}  // namespace ngb
