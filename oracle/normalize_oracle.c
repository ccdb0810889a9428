/*
 * normalize_oracle.c -- the oracle: a plain, slow, single-threaded CPU
 * implementation of the scaling algorithms of W. F. Mascarenhas, "Fast and
 * accurate normalization of vectors and quaternions" (arXiv 1606.06508).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU
 * baseline of the benchmark load this library.  It shares no code, header,
 * constant or helper with the CUDA library; the two meet only on the inputs.
 *
 * What it computes, per vector x of length n (Section 2, Algorithms 3-7):
 *   1. m = max |x_k|; the zero result when every x_k is zero (Scale2D/3D,
 *      Normalize4D);
 *   2. the factor c = 1, sigma_min or sigma_max by comparing m with tau_min
 *      and tau_max (Table 2), and x~ = c x (exact: c is a power of two);
 *   3. r~ = sqrt(x~_1 x~_1 + ... + x~_n x~_n), h = 1/r~;
 *   4. the outputs x^_k = h x~_k and r^ = c^{-1} r~.
 * Every step is one IEEE operation rounded to nearest-even, with no fused
 * multiply-add and no flushing of subnormals (Section 3, remark on DAZ/FTZ).
 *
 * Readings where the paper is silent or garbled (each also listed in the
 * design notes of the repository):
 *   - Table 2's tau_min (2^-49, 2^-482) is used, not the value of Eq. (4);
 *   - Normalize4D's "m <- |x4|" belongs to an omitted Else (as in Scale3D);
 *   - the zero result is returned only when every component compares equal
 *     to zero: as printed, Scale3D and Normalize4D return it for (0, NaN, 0)
 *     and (0, NaN, NaN, 0), against the paper's claim that a NaN input always
 *     gives a NaN output;
 *   - the quaternion zero result [0,0,1,0] is q^ with r^ = 0, and callers
 *     may ask for the all-zero result instead (vector semantics);
 *   - n = 1 runs the Normalize2D steps on one component;
 *   - n >= 5 uses the summation order CR(n) (256 slots) and the constants
 *     tau_max = 2^53 / 2^501, sigma_max = 2^-75 / 2^-523 (binary32 / 64);
 *   - the backward pass (no counterpart in the paper) is
 *     grad = ((g - y (y.g)) * h) * c.
 *
 * Parity unpinned: the n >= 5 summation order CR(n) and the backward
 * operation order are this project's definitions (the paper defines
 * neither).  The tests pin them only by the error bounds, invariants, exact
 * integer norms, finite differences and the exact gradient, which another
 * order within the bounds would pass as well.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#define OR_CODE_ONE 0  /* c = 1         */
#define OR_CODE_SMIN 1 /* c = sigma_min */
#define OR_CODE_SMAX 2 /* c = sigma_max */
#define OR_CODE_ZERO 3 /* x = 0: the zero result, no factor */

#define OR_VECTOR_SEMANTICS 1u /* n = 4: all-zero result for x = 0 */
#define OR_CR_SLOTS 256
#define OR_MAX_LEN (1 << 20)

/* ---- binary32 (Table 2, single precision row) ---- */
#define REAL float
#define SFX(name) name##_f32
#define FABS fabsf
#define SQRT sqrtf
#define COPYSIGN copysignf
#define TAU_MIN 0x1p-49f
#define SIGMA_MIN 0x1p100f
#define INV_SIGMA_MIN 0x1p-100f
#define TAU_MAX 0x1p62f
#define SIGMA_MAX 0x1p-66f
#define INV_SIGMA_MAX 0x1p66f
#define TAU_MAX_N 0x1p53f
#define SIGMA_MAX_N 0x1p-75f
#define INV_SIGMA_MAX_N 0x1p75f
#include "oracle_impl.h"
#undef REAL
#undef SFX
#undef FABS
#undef SQRT
#undef COPYSIGN
#undef TAU_MIN
#undef SIGMA_MIN
#undef INV_SIGMA_MIN
#undef TAU_MAX
#undef SIGMA_MAX
#undef INV_SIGMA_MAX
#undef TAU_MAX_N
#undef SIGMA_MAX_N
#undef INV_SIGMA_MAX_N

/* ---- binary64 (Table 2, double precision row) ---- */
#define REAL double
#define SFX(name) name##_f64
#define FABS fabs
#define SQRT sqrt
#define COPYSIGN copysign
#define TAU_MIN 0x1p-482
#define SIGMA_MIN 0x1p592
#define INV_SIGMA_MIN 0x1p-592
#define TAU_MAX 0x1p510
#define SIGMA_MAX 0x1p-514
#define INV_SIGMA_MAX 0x1p514
#define TAU_MAX_N 0x1p501
#define SIGMA_MAX_N 0x1p-523
#define INV_SIGMA_MAX_N 0x1p523
#include "oracle_impl.h"

/* Returns 1 when the compiled oracle and this thread follow the IEEE model the paper
 * assumes: a product and a sum are rounded separately (no contraction into a
 * fused multiply-add) and subnormal results and operands are kept (no FTZ or
 * DAZ).  The tests refuse to trust the oracle otherwise. */
int oracle_ieee_check(void)
{
    volatile float a = 1.0f + 0x1p-23f, b = 1.0f + 0x1p-23f, c = 1.0f + 0x1p-22f;
    float prod_minus = a * b - c; /* 0 when a*b is rounded before the subtraction */
    volatile double ad = 1.0 + 0x1p-52, bd = 1.0 + 0x1p-52, cd = 1.0 + 0x1p-51;
    double prod_minus_d = ad * bd - cd;
    volatile float tiny = 0x1p-140f, quarter = 0.25f;
    float sub = tiny * quarter; /* 2^-142, subnormal */
    volatile float subin = 0x1p-148f;
    float twice = subin + subin; /* 2^-147, needs subnormal operands */
    volatile double tinyd = 0x1p-1070;
    double subd = tinyd * 0.25;
    return prod_minus == 0.0f && prod_minus_d == 0.0 && sub == 0x1p-142f &&
           twice == 0x1p-147f && subd == 0x1p-1072;
}
