// ngb_f64emu.cuh -- binary64 square, product, sum of non-negative values,
// square root, reciprocal and power-of-two scaling on the integer pipes.
//
// The sum of squares of a vector is a chain of correctly rounded binary64
// multiplications (x~_k * x~_k) and additions (Eq. 3 evaluated left to right
// for n <= 4, in the order CR(n) above), followed by a square root, a
// reciprocal and the output products (Algorithms 5-7).  GB300 executes
// binary64 arithmetic at a small fraction of its integer rate, so these
// operations are rebuilt here from integer products, shifts and adds.  Each returns exactly the IEEE 754 result with
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
#include <math.h>
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

NGB_HD uint32_t funnel_r(uint32_t lo, uint32_t hi, uint32_t n) {  // (hi:lo) >> n, 0 < n < 32
#if defined(__CUDA_ARCH__)
  return __funnelshift_r(lo, hi, n);
#else
  return (uint32_t)((((uint64_t)hi << 32) | lo) >> n);
#endif
}

// a * a for a = |x| (sign bit clear), valid when x = 0, or x is normal and
// its square is normal (square_in_range).
//
// With x = m 2^(e-1075), m = 2^52 + f, the square is m^2 2^(2e-2150) and
// m^2 lies in [2^104, 2^106).  m^2 is formed exactly, as four 32-bit words,
// from three 32 x 32-bit products of m = mh 2^32 + ml:
//     m^2 = mh^2 2^64 + (2 mh ml) 2^32 + ml^2.
// The significand keeps the top 53 bits: k = 52 + s bits are rounded off,
// s = 1 when m^2 >= 2^105, and the biased exponent is 2e - 1023 + s.
// Rounding: a square is never a tie that rounds up (a tie needs
// m^2 = 2^(k-1) o^2 with o odd, and then the last kept bit, bit k, is bit 1
// of o^2, which is 0 because o^2 = 1 (mod 8)), so adding 2^(k-1) - 1 and
// truncating rounds to nearest even.  The low word only contributes its
// carry (w0 != 0) to that addition.  Adding the significand, hidden bit
// included, to (exponent - 1) << 52 packs the result; a rounding carry to
// 2^53 moves into the exponent by itself.
NGB_HD uint64_t square(uint64_t a) {
  const uint32_t hi = (uint32_t)(a >> 32), lo = (uint32_t)a;
  const uint32_t mh = (hi & 0xFFFFFu) | 0x100000u;
  const uint64_t ll = (uint64_t)lo * lo;
  const uint64_t hl2 = (uint64_t)(mh << 1) * lo;  // 2 mh ml < 2^54
  const uint64_t hh = (uint64_t)mh * mh;          // < 2^42
  const uint32_t w0 = (uint32_t)ll;
  const uint64_t t1 = (ll >> 32) + (uint32_t)hl2;
  const uint64_t t2 = (t1 >> 32) + (hl2 >> 32) + (uint32_t)hh;
  const uint32_t w1 = (uint32_t)t1, w2 = (uint32_t)t2;
  const uint32_t w3 = (uint32_t)(t2 >> 32) + (uint32_t)(hh >> 32);  // < 2^10
  const uint32_t s = w3 >> 9;
  const uint64_t u1 = (uint64_t)w1 + ((0x80000u << s) - 1u) + (w0 != 0 ? 1u : 0u);
  const uint64_t u2 = (uint64_t)w2 + (uint32_t)(u1 >> 32);
  const uint32_t v3 = w3 + (uint32_t)(u2 >> 32);
  const uint32_t sh = 20u + s;
  const uint32_t sig_lo = funnel_r((uint32_t)u1, (uint32_t)u2, sh);
  const uint32_t sig_hi = funnel_r((uint32_t)u2, v3, sh);  // < 2^22, hidden bit at 2^20
  const uint32_t e = hi >> 20;
  const uint32_t rhi = sig_hi + ((2u * e + s - 1024u) << 20);
  return e == 0 ? 0 : (((uint64_t)rhi << 32) | sig_lo);
}

// The operands square() takes: x = 0, or x normal with a normal square
// (2^-511 <= |x| < 2^512).
NGB_HD bool square_in_range(uint64_t a) {
  const uint32_t e = (uint32_t)(a >> 52);
  return a == 0 || (e >= 512u && e <= 1534u);
}

// x * y for y > 0, rounded to nearest even, valid when x = +-0 or x and y are
// normal and |x y| is normal without overflow (mul_in_range).  The same word
// arithmetic as square(), with four 32 x 32-bit products
//     mx my = (xh yh) 2^64 + (xh yl + xl yh) 2^32 + xl yl
// and ties possible: the rounding adds 2^(k-1) - 1 + (bit k), which carries
// into bit k exactly when the discarded part is above half a unit, or equal
// to it with bit k odd.  The sign is that of x.
NGB_HD uint64_t mul(uint64_t x, uint64_t y) {
  const uint32_t xh = (uint32_t)(x >> 32), xl = (uint32_t)x;
  const uint32_t yh = (uint32_t)(y >> 32), yl = (uint32_t)y;
  const uint32_t mxh = (xh & 0xFFFFFu) | 0x100000u, myh = (yh & 0xFFFFFu) | 0x100000u;
  const uint64_t ll = (uint64_t)xl * yl;
  const uint64_t lh = (uint64_t)xl * myh;  // < 2^53
  const uint64_t hl = (uint64_t)mxh * yl;  // < 2^53
  const uint64_t hh = (uint64_t)mxh * myh; // < 2^42
  const uint32_t w0 = (uint32_t)ll;
  const uint64_t t1 = (ll >> 32) + (uint32_t)lh + (uint32_t)hl;
  const uint64_t t2 = (t1 >> 32) + (lh >> 32) + (hl >> 32) + (uint32_t)hh;
  const uint32_t w1 = (uint32_t)t1, w2 = (uint32_t)t2;
  const uint32_t w3 = (uint32_t)(t2 >> 32) + (uint32_t)(hh >> 32);  // < 2^10
  const uint32_t s = w3 >> 9;
  const uint32_t sh = 20u + s;
  const uint32_t lsb = (w1 >> sh) & 1u;
  const uint64_t u1 = (uint64_t)w1 + ((0x80000u << s) - 1u) + (lsb | (w0 != 0 ? 1u : 0u));
  const uint64_t u2 = (uint64_t)w2 + (uint32_t)(u1 >> 32);
  const uint32_t v3 = w3 + (uint32_t)(u2 >> 32);
  const uint32_t sig_lo = funnel_r((uint32_t)u1, (uint32_t)u2, sh);
  const uint32_t sig_hi = funnel_r((uint32_t)u2, v3, sh);
  const uint32_t ex = (xh >> 20) & 0x7FFu, ey = yh >> 20;
  const uint32_t rhi = (sig_hi + ((ex + ey + s - 1024u) << 20)) | (xh & 0x80000000u);
  return ex == 0 ? (x & 0x8000000000000000ull) : (((uint64_t)rhi << 32) | sig_lo);
}

// x * y for x, y of either sign: the product of |x| and |y| by mul() with the
// sign x_s XOR y_s; a zero operand gives the signed zero.  Valid when x and
// y are zero or normal with a normal product (mul_in_range on |x|, |y|).
NGB_HD uint64_t mul_signed(uint64_t x, uint64_t y) {
  const uint64_t SIGN = 0x8000000000000000ull;
  const uint64_t s = (x ^ y) & SIGN;
  if ((x << 1) == 0 || (y << 1) == 0) return s;
  return mul(x & ~SIGN, y & ~SIGN) | s;
}

// The operands mul() takes (y > 0): x = +-0, or x and y normal with a normal
// product: the biased exponent ex + ey - 1023 (+1) of x y within [1, 2046].
NGB_HD bool mul_in_range(uint64_t x, uint64_t y) {
  const int ex = (int)((x >> 52) & 0x7FF), ey = (int)(y >> 52);
  if ((x << 1) == 0) return ey != 0 && ey != 0x7FF;
  return ex != 0 && ex != 0x7FF && ey != 0 && ey != 0x7FF && ex + ey - 1023 >= 1 && ex + ey - 1023 <= 2045;
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

// Count of leading zero bits of v != 0.
NGB_HD int clz64(uint64_t v) {
#if defined(__CUDA_ARCH__)
  return __clzll((long long)v);
#else
  return __builtin_clzll(v);
#endif
}

// a + b for finite a, b of either sign (zero and subnormal included), rounded
// to nearest even, when the larger magnitude has a biased exponent of at most
// 2045 (the caller's range test: the sum cannot overflow).
//
// The operands are ordered by magnitude and aligned as in add_nonneg (10
// guard bits, the bits shifted out ORed into bit 0).  Same signs: the
// significands are added as there.  Opposite signs: the smaller is
// subtracted from the larger (the difference is >= 0) and the result is
// shifted left until its leading one is back at bit 62, or until the
// exponent reaches that of 2^-1022 (a subnormal result).  Two cases:
//   - exponent difference 0 or 1: no bit was shifted out, the difference is
//     exact and is only rounded;
//   - difference >= 2: the larger significand has its leading one at bit 62
//     and the aligned smaller one is below 2^61, so the difference keeps its
//     leading one at bit 62 or 61: at most one shift, and at least 9 of the
//     10 guard bits are rounded off.  The exact difference M - A - e
//     (0 < e < 1 in units of bit 0, when bits were lost) lies strictly
//     between two integers; the computed M - (A | 1) is the odd one of them
//     or its odd neighbour below, so no multiple of 2^8 -- a rounding
//     boundary or a tie -- lies between the computed and the exact value, or
//     on the computed one: both round the same way.
// A difference of zero is +0 (round to nearest).
NGB_HD uint64_t add_signed(uint64_t a, uint64_t b) {
  const uint64_t SIGN = uint64_t(1) << 63;
  const uint64_t ma = a & ~SIGN, mbv = b & ~SIGN;
  const bool swap = mbv > ma;
  const uint64_t big = swap ? mbv : ma, small = swap ? ma : mbv;
  const uint64_t sign = (swap ? b : a) & SIGN;
  const int eb = (int)(big >> 52), es = (int)(small >> 52);
  const uint64_t mb = (big & FRAC) | ((uint64_t)(eb != 0 ? 1u : 0u) << 52);
  const uint64_t ms = (small & FRAC) | ((uint64_t)(es != 0 ? 1u : 0u) << 52);
  const int Eb = eb > 1 ? eb : 1;  // subnormals have the exponent of 2^-1022
  const int Es = es > 1 ? es : 1;
  int d = Eb - Es;
  d = d < 63 ? d : 63;
  const uint64_t s10 = ms << 10;
  const uint64_t lost = s10 & ((uint64_t(1) << d) - 1u);
  const uint64_t al = (s10 >> d) | (lost != 0 ? 1u : 0u);
  const uint64_t M = mb << 10;
  if (((a ^ b) & SIGN) == 0) {  // same signs
    const uint64_t sum = M + al;  // < 2^64 - 2^11
    const int c = (int)(sum >> 63);
    const uint64_t sig = round_shift(sum, 10 + c);
    return sign | (((uint64_t)(uint32_t)(Eb - 1 + c) << 52) + sig);
  }
  uint64_t diff = M - al;
  if (diff == 0) return 0;
  const int lz = clz64(diff) - 1;  // shift that puts the leading one at bit 62
  const int sh = lz < Eb - 1 ? lz : Eb - 1;
  diff <<= sh;
  const uint64_t sig = round_shift(diff, 10);
  return sign | (((uint64_t)(uint32_t)(Eb - sh - 1) << 52) + sig);
}

// High 64 bits of the 128-bit product a b.
NGB_HD uint64_t mulhi64(uint64_t a, uint64_t b) {
#if defined(__CUDA_ARCH__)
  return __umul64hi(a, b);
#else
  return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

// Binary32 reciprocal and reciprocal square root, each within a few units in
// its last place.  They only start the Newton iterations below, whose exact
// remainder corrections make the results independent of them.
NGB_HD float approx_rcp(float f) {
#if defined(__CUDA_ARCH__)
  return __frcp_rn(f);
#else
  return 1.0f / f;
#endif
}
NGB_HD float approx_rsqrt(float f) {
#if defined(__CUDA_ARCH__)
  return rsqrtf(f);
#else
  return 1.0f / sqrtf(f);
#endif
}

// RN(1 / r) for r > 0 normal with r < 2^1022 (so that 1/r is normal).
//
// With r = b 2^(e-1075), b = 2^52 + f: 1/r = (2^105 / b) 2^(970-e), and
// 2^105 / b lies in (2^52, 2^53] (= 2^53 only for b = 2^52, where 1/r is a
// power of two).  q = floor(2^105 / b) comes from Newton's iteration
// x <- x (2 - beta x) for x = 1/beta, beta = b 2^11 / 2^64 in [1/2, 1), in
// 64-bit fixed point (X = x 2^63), started from a binary32 reciprocal of the
// top 24 bits of b: two steps take about 22 correct bits to more than 60.
// Then exactly: the remainder 2^105 - q b is small, so it is computed modulo
// 2^64, and q is moved until 0 <= remainder < b.  Round to nearest: up when
// 2 remainder > b; a tie would need b (2q + 1) = 2^106, impossible for q > 0.
// `start_scale` multiplies the binary32 starting point (1 in use; the host
// check perturbs it to show that the correction covers a worse start).
NGB_HD uint64_t rcp_rn(uint64_t r, float start_scale = 1.0f) {
  const uint32_t e = (uint32_t)(r >> 52);
  const uint64_t b = (r & FRAC) | (uint64_t(1) << 52);
  const uint64_t B = b << 11;                          // beta 2^64, in [2^63, 2^64)
  const float f = (float)(uint32_t)(B >> 40);          // top 24 bits, exact in binary32
  float x0 = approx_rcp(f) * 0x1p55f * start_scale;    // x 2^31 = X / 2^32
  x0 = x0 < 4294967295.0f ? x0 : 4294967040.0f;
  uint64_t X = (uint64_t)(uint32_t)x0 << 32;
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const uint64_t P = mulhi64(B, X);   // beta x 2^63
    X = mulhi64(X, 0 - P) << 1;         // x (2 - beta x) 2^63
  }
  uint64_t q = X >> 11;                              // about 2^105 / b
  int64_t rem = (int64_t)(0 - q * b);                // 2^105 - q b (2^105 = 0 modulo 2^64)
#pragma unroll
  for (int it = 0; it < 3; ++it)
    if (rem < 0) { q -= 1; rem += (int64_t)b; }
#pragma unroll
  for (int it = 0; it < 3; ++it)
    if (rem >= (int64_t)b) { q += 1; rem -= (int64_t)b; }
  q += (uint64_t)(2 * rem > (int64_t)b ? 1 : 0);
  if (b == (uint64_t(1) << 52)) q = uint64_t(1) << 53;  // 1/r is a power of two
  // q in [2^52, 2^53]: adding it (hidden bit included) to (2044 - e) << 52
  // gives the biased exponent 2045 - e, or 2046 - e when q = 2^53
  return ((uint64_t)(2044u - e) << 52) + q;
}

// RN(sqrt(s)) for s > 0 normal.
//
// With s = (m / 2^52) 2^E, m = 2^52 + f: make the exponent even (M = m 2^odd,
// odd = E mod 2), so that sqrt(s) = sqrt(M 2^52) 2^(Eh - 52), Eh = (E - odd) / 2,
// and q = floor(sqrt(M 2^52)) lies in [2^52, 2^53).  q comes from Newton's
// iteration y <- y (3 - mu y^2) / 2 for y = 1/sqrt(mu), mu = M / 2^54 in
// [1/4, 1), in 64-bit fixed point (Y = y 2^62), started from a binary32
// reciprocal square root of the top 24 bits of M; then q ~ mu y 2^53.  Then
// exactly: the remainder M 2^52 - q^2 is small, so it is computed modulo
// 2^64, and q is moved until 0 <= remainder <= 2q.  Round to nearest: up when
// remainder > q, since (q + 1/2)^2 = q^2 + q + 1/4; no tie is possible.
NGB_HD uint64_t sqrt_rn(uint64_t s, float start_scale = 1.0f) {
  const uint32_t e = (uint32_t)(s >> 52);
  const uint64_t m = (s & FRAC) | (uint64_t(1) << 52);
  const int E = (int)e - 1023;
  const uint32_t odd = (uint32_t)E & 1u;
  const uint64_t M = m << odd;                         // [2^52, 2^54)
  const int Eh = (E - (int)odd) / 2;                   // exact: E - odd is even
  const uint64_t Mq = M << 10;                         // mu 2^64
  const float f = (float)(uint32_t)(M >> 30);          // top 24 bits, exact in binary32
  float y0 = approx_rsqrt(f) * 0x1p42f * start_scale;  // y 2^30 = Y / 2^32
  y0 = y0 < 4294967295.0f ? y0 : 4294967040.0f;
  uint64_t Y = (uint64_t)(uint32_t)y0 << 32;
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const uint64_t Y2 = mulhi64(Y, Y);                 // y^2 2^60
    const uint64_t T = mulhi64(Mq, Y2);                // mu y^2 2^60
    const uint64_t D = (uint64_t(3) << 60) - T;        // (3 - mu y^2) 2^60
    Y = mulhi64(Y, D << 2) << 1;                       // y (3 - mu y^2) / 2 2^62
  }
  uint64_t q = mulhi64(Mq, Y) >> 9;                    // mu y 2^53, about sqrt(M 2^52)
  int64_t rem = (int64_t)((M << 52) - q * q);          // M 2^52 - q^2, modulo 2^64
#pragma unroll
  for (int it = 0; it < 3; ++it)
    if (rem < 0) { rem += (int64_t)(2 * q - 1); q -= 1; }
#pragma unroll
  for (int it = 0; it < 3; ++it)
    if (rem > (int64_t)(2 * q)) { q += 1; rem -= (int64_t)(2 * q - 1); }
  q += (uint64_t)(rem > (int64_t)q ? 1 : 0);
  // q in [2^52, 2^53]: the hidden bit (or the carry to 2^53) completes the exponent
  return ((uint64_t)(uint32_t)(Eh + 1022) << 52) + q;
}

// RN(a 2^d) for a > 0 normal.  A normal result is exact: the exponent field
// moves by d.  Above the largest finite value the exact product is at least
// 2^1024 and rounds to +infinity.  Below 2^-1022 the result counts units of
// 2^-1074: the significand m (hidden bit included) divided by 2^k,
// k = 1 - (biased exponent + d), rounded to nearest even; a carry to 2^52
// gives the smallest normal number by itself.
NGB_HD uint64_t ldexp_rn(uint64_t a, int d) {
  const int ne = (int)(a >> 52) + d;
  if (ne >= 2047) return 0x7FF0000000000000ull;
  if (ne >= 1) return (uint64_t)((int64_t)a + (int64_t)d * (int64_t(1) << 52));
  const int k = 1 - ne < 63 ? 1 - ne : 63;
  return round_shift((a & FRAC) | (uint64_t(1) << 52), k);
}

}  // namespace f64emu
}  // namespace ngb
