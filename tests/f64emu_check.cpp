// Host check of the integer-pipe binary64 square, product, sums, square root,
// reciprocal and power-of-two scaling (csrc/ngb_f64emu.cuh) against the host's
// IEEE 754 binary64 multiply, add, divide and square root (round to nearest
// even).  Prints "<cases> <in range> <mismatches>" per operation; any mismatch
// on an operand the routine takes is a failure.  Built with -ffp-contract=off.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "ngb_f64emu.cuh"

static uint64_t sm_state;
static uint64_t next64() {  // splitmix64
  uint64_t z = (sm_state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
static uint64_t bits(double x) { uint64_t b; std::memcpy(&b, &x, 8); return b; }
static double val(uint64_t b) { double x; std::memcpy(&x, &b, 8); return x; }

// a non-negative finite value with biased exponent e and a fraction that is
// random, all ones, all zeros or has few bits set
static uint64_t make(int e, int kind) {
  uint64_t f = next64() & ngb::f64emu::FRAC;
  if (kind == 1) f = ngb::f64emu::FRAC;
  if (kind == 2) f = 0;
  if (kind == 3) f &= next64() & next64() & next64();
  if (kind == 4) f = ngb::f64emu::FRAC - (next64() & 0xFF);
  if (kind == 5) f = (f & ~((uint64_t(1) << 27) - 1u)) | (uint64_t(1) << 26);  // m = 2^26 odd: square ties
  return ((uint64_t)e << 52) | f;
}

int main(int argc, char** argv) {
  const long n = argc > 1 ? atol(argv[1]) : 1000000;
  sm_state = argc > 2 ? strtoull(argv[2], 0, 10) : 1;
  long sq_fast = 0, sq_bad = 0, add_fast = 0, add_bad = 0;
  for (long i = 0; i < n; ++i) {
    const int kind = (int)(next64() % 6);
    // exponents: uniform, or close to the edges of the fast path
    int e;
    const int sel = (int)(next64() % 4);
    if (sel == 0) e = (int)(next64() % 2047);
    else if (sel == 1) e = 509 + (int)(next64() % 6);   // squares near 2^-1022
    else if (sel == 2) e = 1532 + (int)(next64() % 6);  // squares near 2^1024
    else e = 1023 + (int)(next64() % 64) - 32;
    const uint64_t a = make(e, kind);
    bool ok = ngb::f64emu::square_in_range(a);
    const uint64_t r = ngb::f64emu::square(a);
    if (ok) {
      ++sq_fast;
      const double x = val(a);
      if (r != bits(x * x)) {
        if (sq_bad < 5) fprintf(stderr, "square %016llx: %016llx vs %016llx\n", (unsigned long long)a,
                                (unsigned long long)r, (unsigned long long)bits(x * x));
        ++sq_bad;
      }
    }
    // sums: the second operand d binades below the first (d in [-2, 70]),
    // or a subnormal, zero, or a value that makes a tie
    const int eb = (int)(next64() % 2048) % 2046;
    const int mode = (int)(next64() % 5);
    uint64_t p = make(eb, kind), q;
    if (mode == 0) {
      int d = (int)(next64() % 73) - 2;
      int es = eb - d;
      if (es < 0) es = 0;
      if (es > 2045) es = 2045;
      q = make(es, (int)(next64() % 6));
    } else if (mode == 1) {
      q = next64() & ngb::f64emu::FRAC;  // subnormal or zero
      if (next64() & 1) p = next64() & ngb::f64emu::FRAC;
    } else if (mode == 2) {
      q = 0;
    } else if (mode == 3) {  // q = half an ulp of p (and neighbours): ties
      int es = eb - 53;
      if (es < 1) es = 1;
      q = ((uint64_t)es << 52) | ((next64() % 3 == 0) ? 0 : (next64() & 1));
    } else {
      q = make(eb, (int)(next64() % 6));  // same binade: carry and normalisation
    }
    if (next64() & 1) { const uint64_t t = p; p = q; q = t; }
    const uint64_t s = ngb::f64emu::add_nonneg(p, q, ok);
    if (ok) {
      ++add_fast;
      const double ref = val(p) + val(q);
      if (s != bits(ref)) {
        if (add_bad < 5) fprintf(stderr, "add %016llx + %016llx: %016llx vs %016llx\n", (unsigned long long)p,
                                 (unsigned long long)q, (unsigned long long)s, (unsigned long long)bits(ref));
        ++add_bad;
      }
    }
  }
  // signed sums: operands of either sign, d binades apart (d in [-2, 70]),
  // equal magnitudes, one-ulp neighbours (cancellation down to the last bit),
  // subnormals and zeros of either sign, half-ulp ties; larger exponent <= 2045
  long sadd_bad = 0;
  for (long i = 0; i < n; ++i) {
    const int eb = (int)(next64() % 2046);
    const int mode = (int)(next64() % 6);
    uint64_t p = make(eb, (int)(next64() % 6)), q;
    if (mode == 0) {
      int es = eb - ((int)(next64() % 73) - 2);
      es = es < 0 ? 0 : (es > 2045 ? 2045 : es);
      q = make(es, (int)(next64() % 6));
    } else if (mode == 1) {
      q = next64() & ngb::f64emu::FRAC;
      if (next64() & 1) p = next64() & ngb::f64emu::FRAC;
    } else if (mode == 2) {
      q = (next64() & 1) ? 0 : p;
    } else if (mode == 3) {
      q = p + (uint64_t)((int)(next64() % 5) - 2);  // neighbours: massive cancellation
      if ((q >> 52) > 2045) q = p;
    } else if (mode == 4) {
      int es = eb - 53 + (int)(next64() % 3) - 1;
      if (es < 1) es = 1;
      q = ((uint64_t)es << 52) | ((next64() % 3 == 0) ? 0 : (next64() & 1));
    } else {
      q = make(eb, (int)(next64() % 6));
    }
    if (next64() & 1) p |= uint64_t(1) << 63;
    if (next64() & 1) q |= uint64_t(1) << 63;
    if (next64() & 1) { const uint64_t t = p; p = q; q = t; }
    const uint64_t s = ngb::f64emu::add_signed(p, q);
    const double ref = val(p) + val(q);
    if (s != bits(ref)) {
      if (sadd_bad < 5) fprintf(stderr, "add_signed %016llx + %016llx: %016llx vs %016llx\n", (unsigned long long)p,
                                (unsigned long long)q, (unsigned long long)s, (unsigned long long)bits(ref));
      ++sadd_bad;
    }
  }
  long mul_fast = 0, mul_bad = 0;
  for (long i = 0; i < n; ++i) {  // products: x of either sign, y > 0, exponents near the limits too
    const int sel = (int)(next64() % 4);
    int ex, ey;
    if (sel == 0) { ex = 1 + (int)(next64() % 2045); ey = 1 + (int)(next64() % 2045); }
    else if (sel == 1) { ex = 1 + (int)(next64() % 40); ey = 1023 - 40 + (int)(next64() % 80); }  // near 2^-1022
    else if (sel == 2) { ex = 512 + (int)(next64() % 8); ey = 512 + (int)(next64() % 8); }
    else { ex = 1023 + (int)(next64() % 64) - 32; ey = 1023 + (int)(next64() % 64) - 32; }
    uint64_t x = make(ex, (int)(next64() % 6)), y = make(ey, (int)(next64() % 6));
    if (next64() % 16 == 0) x = 0;
    if (next64() & 1) x |= uint64_t(1) << 63;
    if (ngb::f64emu::mul_in_range(x, y)) {
      ++mul_fast;
      const uint64_t r = ngb::f64emu::mul(x, y);
      const double ref = val(x) * val(y);
      if (r != bits(ref)) {
        if (mul_bad < 5) fprintf(stderr, "mul %016llx * %016llx: %016llx vs %016llx\n", (unsigned long long)x,
                                 (unsigned long long)y, (unsigned long long)r, (unsigned long long)bits(ref));
        ++mul_bad;
      }
    }
  }
  long smul_fast = 0, smul_bad = 0;
  for (long i = 0; i < n; ++i) {  // signed products, zeros of either sign included
    int ex = 1023 + (int)(next64() % 200) - 100, ey = 1023 + (int)(next64() % 200) - 100;
    if (next64() % 8 == 0) { ex = 1 + (int)(next64() % 30); ey = 1023 - 30 + (int)(next64() % 60); }
    uint64_t x = make(ex, (int)(next64() % 6)), y = make(ey, (int)(next64() % 6));
    if (next64() % 16 == 0) x = 0;
    if (next64() % 16 == 0) y = 0;
    if (next64() & 1) x |= uint64_t(1) << 63;
    if (next64() & 1) y |= uint64_t(1) << 63;
    const uint64_t ax = x & ~(uint64_t(1) << 63), ay = y & ~(uint64_t(1) << 63);
    const bool zero = (ax == 0) || (ay == 0);
    if (zero || (ngb::f64emu::mul_in_range(ax, ay) && ((ay >> 52) != 0))) {
      ++smul_fast;
      const uint64_t r = ngb::f64emu::mul_signed(x, y);
      const double ref = val(x) * val(y);
      if (r != bits(ref)) {
        if (smul_bad < 5) fprintf(stderr, "mul_signed %016llx * %016llx: %016llx vs %016llx\n", (unsigned long long)x,
                                  (unsigned long long)y, (unsigned long long)r, (unsigned long long)bits(ref));
        ++smul_bad;
      }
    }
  }
  // square roots and reciprocals of normal values, with perturbed binary32
  // starting points (the device's are within a few units of binary32), plus
  // exact squares and powers of two
  long sr_cases = 0, sr_bad = 0, rc_cases = 0, rc_bad = 0;
  const float scales[5] = {1.0f, 1.0f + 0x1p-18f, 1.0f - 0x1p-18f, 1.0f + 0x1p-21f, 1.0f - 0x1p-21f};
  for (long i = 0; i < n; ++i) {
    int e = 1 + (int)(next64() % 2046);
    if (next64() % 4 == 0) e = 1023 + (int)(next64() % 40) - 20;
    if (next64() % 16 == 0) e = (next64() & 1) ? 1 + (int)(next64() % 3) : 2046 - (int)(next64() % 3);
    uint64_t a = make(e, (int)(next64() % 6));
    if (next64() % 8 == 0) {  // an exact square j^2 2^(2t), or its neighbours
      const uint64_t j = (next64() >> 38) | 1u;  // odd, < 2^26
      const double sq = (double)j * (double)j;   // exact: < 2^52
      const int t = (int)(next64() % 800) - 400;
      a = bits(std::ldexp(sq, 2 * t)) + (uint64_t)((int)(next64() % 3) - 1);
    }
    const float sc = scales[next64() % 5];
    ++sr_cases;
    const uint64_t r = ngb::f64emu::sqrt_rn(a, sc);
    if (r != bits(std::sqrt(val(a)))) {
      if (sr_bad < 5) fprintf(stderr, "sqrt %016llx: %016llx vs %016llx\n", (unsigned long long)a,
                              (unsigned long long)r, (unsigned long long)bits(std::sqrt(val(a))));
      ++sr_bad;
    }
    if ((a >> 52) <= 2044) {  // r < 2^1022
      ++rc_cases;
      const uint64_t h = ngb::f64emu::rcp_rn(a, sc);
      if (h != bits(1.0 / val(a))) {
        if (rc_bad < 5) fprintf(stderr, "rcp %016llx: %016llx vs %016llx\n", (unsigned long long)a,
                                (unsigned long long)h, (unsigned long long)bits(1.0 / val(a)));
        ++rc_bad;
      }
    }
  }
  // a 2^d for d in [-1022, 1023] (so that 2^d is a normal binary64 value and
  // the reference is one IEEE multiplication), results from subnormal to
  // infinite
  long ld_bad = 0;
  for (long i = 0; i < n; ++i) {
    const int e = 1 + (int)(next64() % 2046);
    const uint64_t a = make(e, (int)(next64() % 6));
    int d = (int)(next64() % 2046) - 1022;
    if (next64() & 1) d = (1 - e) - (int)(next64() % 56) + 2;  // near and below 2^-1022
    if (d < -1022) d = -1022;
    if (d > 1023) d = 1023;
    const uint64_t r = ngb::f64emu::ldexp_rn(a, d);
    const double ref = val(a) * std::ldexp(1.0, d);
    if (r != bits(ref)) {
      if (ld_bad < 5) fprintf(stderr, "ldexp %016llx %d: %016llx vs %016llx\n", (unsigned long long)a, d,
                              (unsigned long long)r, (unsigned long long)bits(ref));
      ++ld_bad;
    }
  }
  printf("sqrt %ld %ld %ld\n", n, sr_cases, sr_bad);
  printf("rcp %ld %ld %ld\n", n, rc_cases, rc_bad);
  printf("ldexp %ld %ld %ld\n", n, n, ld_bad);
  printf("square %ld %ld %ld\n", n, sq_fast, sq_bad);
  printf("mul_signed %ld %ld %ld\n", n, smul_fast, smul_bad);
  printf("mul %ld %ld %ld\n", n, mul_fast, mul_bad);
  printf("add %ld %ld %ld\n", n, add_fast, add_bad);
  printf("add_signed %ld %ld %ld\n", n, n, sadd_bad);
  return (sq_bad || add_bad || sadd_bad || mul_bad || smul_bad || sr_bad || rc_bad || ld_bad) ? 1 : 0;
}
