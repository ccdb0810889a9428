// Host stand-ins for the CUDA qualifiers and arithmetic intrinsics that the
// kernels' arithmetic uses, shared by the two host builds of the kernel
// sources in tests/: the __*_rn intrinsics are the host's IEEE 754
// operations, round to nearest even (the tests build with -ffp-contract=off,
// so nothing is fused); bit casts go through memcpy.
#pragma once
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cmath>

#define __device__
#define __host__
#define __forceinline__ inline
#define __noinline__
#define __restrict__

using std::max;
using std::min;

inline float __fmul_rn(float a, float b) { return a * b; }
inline float __fadd_rn(float a, float b) { return a + b; }
inline float __fsub_rn(float a, float b) { return a - b; }
inline float __fdiv_rn(float a, float b) { return a / b; }
inline float __fsqrt_rn(float a) { return std::sqrt(a); }
inline float __frcp_rn(float a) { return 1.0f / a; }
inline double __dmul_rn(double a, double b) { return a * b; }
inline double __dadd_rn(double a, double b) { return a + b; }
inline double __dsub_rn(double a, double b) { return a - b; }
inline double __ddiv_rn(double a, double b) { return a / b; }
inline double __dsqrt_rn(double a) { return std::sqrt(a); }
inline double __drcp_rn(double a) { return 1.0 / a; }
inline float rsqrtf(float a) { return 1.0f / std::sqrt(a); }

inline long long __double_as_longlong(double v) {
  long long b;
  memcpy(&b, &v, sizeof b);
  return b;
}
inline double __longlong_as_double(long long b) {
  double v;
  memcpy(&v, &b, sizeof v);
  return v;
}

