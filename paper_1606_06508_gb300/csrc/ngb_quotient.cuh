// ngb_quotient.cuh -- the quotient algorithms that Mascarenhas (arXiv
// 1606.06508, Section 1) compares the scaling algorithms with, for three
// components: Algorithm 1 (robust quotient algorithm) and Algorithm 2 (fast
// robust quotient algorithm).  Not the method: built to measure the paper's
// Table 3 ratio time(quotient) / time(scaling) on the GPU.  Every step is one
// correctly rounded IEEE operation (divisions by __fdiv_rn / __ddiv_rn).
#pragma once
#include "ngb_arith.cuh"

namespace ngb {

// Algorithm 1: m = max |x_k| (a NaN never compares greater); m = 0 returns
// r = 0 and x unchanged; otherwise t_k = x_k / m, r = m sqrt(t1^2 + t2^2 +
// t3^2), outputs x_k / r (the input components: dividing the scaled t_k by r
// would give x_k / (m r)).
template <typename T>
__device__ __forceinline__ void quotient1_3(const T (&x)[3], T (&y)[3], T& r) {
  using F = FP<T>;
  T m = F::abs(x[0]);
  if (F::abs(x[1]) > m) m = F::abs(x[1]);
  if (F::abs(x[2]) > m) m = F::abs(x[2]);
  if (m == T(0)) {
    r = T(0);
    y[0] = x[0];
    y[1] = x[1];
    y[2] = x[2];
    return;
  }
  const T t1 = F::div(x[0], m), t2 = F::div(x[1], m), t3 = F::div(x[2], m);
  r = F::mul(m, F::sqrt(F::add(F::add(F::mul(t1, t1), F::mul(t2, t2)), F::mul(t3, t3))));
  y[0] = F::div(x[0], r);
  y[1] = F::div(x[1], r);
  y[2] = F::div(x[2], r);
}

// Lines 3-7 of Algorithm 2 with pivot xp and the other two components a, b in
// the roles of x1, x2: q1 = a / xp, q2 = b / xp, h = sqrt(1 + q1^2 + q2^2),
// r = |xp| h, s = sign(xp) / h; outputs q1 s, q2 s, s.
template <typename T>
__device__ __forceinline__ void quotient2_pivot(T xp, T a, T b, T& r, T& yp, T& ya, T& yb) {
  using F = FP<T>;
  const T q1 = F::div(a, xp), q2 = F::div(b, xp);
  const T h = F::sqrt(F::add(F::add(T(1), F::mul(q1, q1)), F::mul(q2, q2)));
  r = F::mul(F::abs(xp), h);
  const T s = F::div(copysign(T(1), xp), h);
  ya = F::mul(q1, s);
  yb = F::mul(q2, s);
  yp = s;
}

// Algorithm 2, branch by branch (pivot = the component of largest
// magnitude; the zero return needs x1 = x3 = 0, so that a NaN input gives NaN
// outputs as the paper states).
template <typename T>
__device__ __forceinline__ void quotient2_3(const T (&x)[3], T (&y)[3], T& r) {
  using F = FP<T>;
  const T x1 = x[0], x2 = x[1], x3 = x[2];
  if (F::abs(x1) > F::abs(x2)) {
    if (F::abs(x3) > F::abs(x1)) quotient2_pivot(x3, x1, x2, r, y[2], y[0], y[1]);
    else quotient2_pivot(x1, x3, x2, r, y[0], y[2], y[1]);
  } else {
    if (F::abs(x3) >= F::abs(x2)) {
      if (x3 == T(0) && x1 == T(0)) {
        r = T(0);
        y[0] = T(0);
        y[1] = T(0);
        y[2] = T(0);
        return;
      }
      quotient2_pivot(x3, x1, x2, r, y[2], y[0], y[1]);
    } else {
      quotient2_pivot(x2, x1, x3, r, y[1], y[0], y[2]);
    }
  }
}

}  // namespace ngb
