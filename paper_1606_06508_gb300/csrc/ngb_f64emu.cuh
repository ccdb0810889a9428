// ngb_f64emu.cuh -- binary64 square and sum of non-negative values on the
// integer pipes.
//
// The sum of squares of a long vector is a chain of correctly rounded binary64
// multiplications (x~_k * x~_k) and additions (Eq. 3 evaluated in the order
// CR(n)).  GB300 executes binary64 arithmetic at a small fraction of its
// integer rate, so these two operations are rebuilt here from 32-bit integer
// products, shifts and adds.  Each returns exactly the IEEE 754 result with
// round to nearest, ties to even, of the operation it replaces, on the
// operands it accepts; on any other operand it clears `ok` and the caller
// uses the hardware instruction instead.  Only the rounding rule of IEEE 754
// is used: the result is the representable value nearest to the exact one,
// and of two equally near ones the one with an even significand.
//
// Values travel as their bit patterns (uint64_t); every operand here is
// non-negative (a square or a sum of squares), so the sign bit is zero and
// the bit patterns of finite values order like the values.
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define NGB_HD __host__ __device__ __forceinline__
#else
#define NGB_HD inline
#endif

namespace ngb {
namespace f64emu {

constexpr uint64_t FRAC = (uint64_t(1) << 52) - 1;

// RNE of the integer v to v >> k (1 <= k <= 63), given that v + 2^(k-1) does
// not wrap: adding 2^(k-1) - 1 + (bit k of v) carries into bit k exactly when
// the discarded part exceeds half a unit, or equals it with bit k odd.
NGB_HD uint64_t round_shift(uint64_t v, int k) {
  const uint64_t lsb = (v >> k) & 1u;
  return (v + ((uint64_t(1) << (k - 1)) - 1u) + lsb) >> k;
}

// a * a for a = |x| (sign bit clear).  Fast path: x normal and the square
// normal without overflow (biased exponent of the square in [1, 2046]).
//
// With x = m 2^(e-1075), m = 2^52 + f, the square is m^2 2^(2e-2150) and
// m^2 lies in [2^104, 2^106).  m^2 is formed exactly from three 32 x 32-bit
// products of m = mh 2^32 + ml:  m^2 = mh^2 2^64 + (mh ml) 2^33 + ml^2.
// The significand keeps the top 53 bits (k = 52 or 53 bits are rounded off)
// and the biased exponent is 2e - 1023 (k = 52) or 2e - 1022 (k = 53).
// Adding the significand, hidden bit included, to (exponent - 1) << 52 packs
// the result; a rounding carry to 2^53 moves into the exponent by itself.
// A square is never a tie that rounds up: a tie needs k = 53 and m = 2^26 o
// with o odd, and then the last kept place, bit 53 of m^2 = 2^52 o^2, is bit 1
// of o^2, which is 0 because o^2 = 1 (mod 8).  So adding 2^(k-1) - 1 and
// truncating rounds to nearest even.
NGB_HD uint64_t square(uint64_t a, bool& ok) {
  const int e = (int)(a >> 52);
  const uint32_t ml = (uint32_t)a;
  const uint32_t mh = ((uint32_t)(a >> 32) & 0xFFFFFu) | 0x100000u;
  const uint64_t ll = (uint64_t)ml * ml;
  const uint64_t hl = (uint64_t)mh * ml;
  const uint64_t hh = (uint64_t)mh * mh;
  const uint64_t L = ll + (hl << 33);
  uint64_t H = hh + (hl >> 31) + (L < ll ? 1u : 0u);  // H < 2^42
  const int s = (int)(H >> 41);                        // m^2 >= 2^105
  const int k = 52 + s;
  // round (H, L) >> k: k <= 53, so the rounding increment touches L only
  const uint64_t L2 = L + ((uint64_t(1) << (k - 1)) - 1u);
  H += (L2 < L ? 1u : 0u);
  const uint64_t sig = (H << (64 - k)) | (L2 >> k);  // in [2^52, 2^53]
  const int E0 = 2 * e - 1024 + s;                   // biased exponent - 1
  ok = (e != 0) && (E0 >= 0) && (E0 <= 2044);
  return ((uint64_t)(uint32_t)E0 << 52) + sig;
}

// a + b for non-negative finite a, b (zero and subnormal included).  Fast
// path: the larger operand has a biased exponent of at most 2045, so the sum
// is finite or rounds to +infinity exactly as IEEE prescribes.
//
// Both significands are placed 10 bits up in a 64-bit word (53 + 10 bits,
// one bit of headroom for the carry); the smaller one is shifted right by the
// exponent difference d with the bits shifted out ORed into bit 0 (sticky).
// With 10 guard bits below the result's last place, that single sticky bit
// decides every tie correctly.  The sum is then rounded off by 10 bits, or by
// 11 when it carried into bit 63.
NGB_HD uint64_t add_nonneg(uint64_t a, uint64_t b, bool& ok) {
  const bool swap = b > a;
  const uint64_t big = swap ? b : a, small = swap ? a : b;
  const int eb = (int)(big >> 52), es = (int)(small >> 52);
  const uint64_t mb = (big & FRAC) | ((uint64_t)(eb != 0 ? 1u : 0u) << 52);
  const uint64_t ms = (small & FRAC) | ((uint64_t)(es != 0 ? 1u : 0u) << 52);
  const int Eb = eb > 1 ? eb : 1;  // subnormals have the exponent of 2^-1022
  const int Es = es > 1 ? es : 1;
  int d = Eb - Es;
  d = d < 63 ? d : 63;  // ms 2^10 < 2^63: a shift by 63 leaves only the sticky bit
  const uint64_t s10 = ms << 10;
  const uint64_t lost = s10 & ((uint64_t(1) << d) - 1u);
  const uint64_t al = (s10 >> d) | (lost != 0 ? 1u : 0u);
  const uint64_t sum = (mb << 10) + al;  // < 2^64 - 2^11
  const int c = (int)(sum >> 63);
  const uint64_t sig = round_shift(sum, 10 + c);
  ok = eb <= 2045;
  return ((uint64_t)(uint32_t)(Eb - 1 + c) << 52) + sig;
}

}  // namespace f64emu
}  // namespace ngb
