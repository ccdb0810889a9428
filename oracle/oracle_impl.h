/*
 * oracle_impl.h -- one binary format of the oracle.  TEST INFRASTRUCTURE ONLY.
 *
 * Included twice by normalize_oracle.c, once with REAL = float and once with
 * REAL = double.  The includer defines:
 *   REAL, SFX(name)        the floating type and the name suffix (_f32 / _f64)
 *   FABS, SQRT             fabsf/sqrtf or fabs/sqrt (IEEE, correctly rounded)
 *   TAU_MIN, SIGMA_MIN, TAU_MAX, SIGMA_MAX          Table 2 of the paper (n <= 4)
 *   INV_SIGMA_MIN, INV_SIGMA_MAX                    their exact inverses
 *   TAU_MAX_N, SIGMA_MAX_N, INV_SIGMA_MAX_N         the constants for 5 <= n <= 2^20
 *
 * Every arithmetic operation below is one IEEE operation in REAL, rounded to
 * nearest-even.  The file is compiled with -ffp-contract=off (no fused
 * multiply-add) and runs with flush-to-zero and denormals-are-zero off, as
 * the paper's error analysis assumes (Section 3, remark on DAZ/FTZ).  C
 * evaluates a + b + c as (a + b) + c, which is the order of the sums printed
 * in Algorithms 5, 6 and 7.
 *
 * Naming follows the paper: x are the inputs, x~ (t[] here) the scaled
 * inputs, sigma the INVERSE of the factor applied to x (the first value
 * returned by Scale2D/Scale3D), r~ (rt) the norm of the scaled vector,
 * h = 1/r~, and the returned pair [sigma * r~, h * x~].
 */

/* ---------------------------------------------------------------------- */
/* Algorithm 3 (Scale2D).  Returns the factor code and writes sigma and x~.  */
static int SFX(scale2)(REAL x1, REAL x2, REAL *sigma, REAL t[2])
{
    REAL m = FABS(x1);
    if (m >= FABS(x2)) {
        if (m == 0) { *sigma = 0; t[0] = 0; t[1] = 0; return OR_CODE_ZERO; }
    } else {
        m = FABS(x2);
    }
    if (m >= TAU_MIN) {
        if (m <= TAU_MAX) { *sigma = 1; t[0] = x1; t[1] = x2; return OR_CODE_ONE; }
        *sigma = INV_SIGMA_MAX;
        t[0] = SIGMA_MAX * x1; t[1] = SIGMA_MAX * x2;
        return OR_CODE_SMAX;
    }
    *sigma = INV_SIGMA_MIN;
    t[0] = SIGMA_MIN * x1; t[1] = SIGMA_MIN * x2;
    return OR_CODE_SMIN;
}

/* Algorithm 4 (Scale3D). */
static int SFX(scale3)(REAL x1, REAL x2, REAL x3, REAL *sigma, REAL t[3])
{
    REAL m = FABS(x1);
    if (m < FABS(x2)) {
        m = FABS(x2);
        if (m < FABS(x3)) m = FABS(x3);
    } else {
        if (m >= FABS(x3)) {
            /* m = 0 here leaves x2 zero or NaN: the zero result only for x2 = 0,
             * so that a NaN input always gives NaN outputs (Section 2). */
            if (m == 0 && x2 == 0) { *sigma = 0; t[0] = 0; t[1] = 0; t[2] = 0; return OR_CODE_ZERO; }
        } else {
            m = FABS(x3);
        }
    }
    if (m >= TAU_MIN) {
        if (m <= TAU_MAX) { *sigma = 1; t[0] = x1; t[1] = x2; t[2] = x3; return OR_CODE_ONE; }
        *sigma = INV_SIGMA_MAX;
        t[0] = SIGMA_MAX * x1; t[1] = SIGMA_MAX * x2; t[2] = SIGMA_MAX * x3;
        return OR_CODE_SMAX;
    }
    *sigma = INV_SIGMA_MIN;
    t[0] = SIGMA_MIN * x1; t[1] = SIGMA_MIN * x2; t[2] = SIGMA_MIN * x3;
    return OR_CODE_SMIN;
}

/* One-component vectors: Scale2D with the second component absent.  The
 * paper does not treat n = 1; this is the reading used for it. */
static int SFX(scale1)(REAL x1, REAL *sigma, REAL t[1])
{
    REAL m = FABS(x1);
    if (m == 0) { *sigma = 0; t[0] = 0; return OR_CODE_ZERO; }
    if (m >= TAU_MIN) {
        if (m <= TAU_MAX) { *sigma = 1; t[0] = x1; return OR_CODE_ONE; }
        *sigma = INV_SIGMA_MAX; t[0] = SIGMA_MAX * x1; return OR_CODE_SMAX;
    }
    *sigma = INV_SIGMA_MIN; t[0] = SIGMA_MIN * x1; return OR_CODE_SMIN;
}

/* ---------------------------------------------------------------------- */
/* n = 1, the Normalize2D steps on one component. */
static int SFX(normalize1)(const REAL *x, REAL *y, REAL *r, REAL *hout)
{
    REAL sigma, t[1];
    int code = SFX(scale1)(x[0], &sigma, t);
    if (sigma == 0) { y[0] = 0; *r = 0; *hout = 0; return code; }
    REAL rt = SQRT(t[0] * t[0]);
    REAL h = 1 / rt;
    *r = sigma * rt;
    y[0] = h * t[0];
    *hout = h;
    return code;
}

/* Algorithm 5 (Normalize2D). */
static int SFX(normalize2)(const REAL *x, REAL *y, REAL *r, REAL *hout)
{
    REAL sigma, t[2];
    int code = SFX(scale2)(x[0], x[1], &sigma, t);
    if (sigma == 0) { y[0] = 0; y[1] = 0; *r = 0; *hout = 0; return code; }
    REAL rt = SQRT(t[0] * t[0] + t[1] * t[1]);
    REAL h = 1 / rt;
    *r = sigma * rt;
    y[0] = h * t[0];
    y[1] = h * t[1];
    *hout = h;
    return code;
}

/* Algorithm 6 (Normalize3D). */
static int SFX(normalize3)(const REAL *x, REAL *y, REAL *r, REAL *hout)
{
    REAL sigma, t[3];
    int code = SFX(scale3)(x[0], x[1], x[2], &sigma, t);
    if (sigma == 0) { y[0] = 0; y[1] = 0; y[2] = 0; *r = 0; *hout = 0; return code; }
    REAL rt = SQRT(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
    REAL h = 1 / rt;
    *r = sigma * rt;
    y[0] = h * t[0];
    y[1] = h * t[1];
    y[2] = h * t[2];
    *hout = h;
    return code;
}

/* Algorithm 7 (Normalize4D).  The branch at "m >= |x4|" takes the reading in
 * which the assignment m <- |x4| belongs to an omitted Else, as in Scale3D;
 * read literally, it would replace the maximum by a smaller value.  The zero
 * quaternion gives [0, 0, 1, 0] with r = 0 when quat_zero is set, and the
 * zero vector otherwise. */
static int SFX(normalize4)(const REAL *x, REAL *y, REAL *r, REAL *hout, int quat_zero)
{
    REAL x1 = x[0], x2 = x[1], x3 = x[2], x4 = x[3];
    REAL sigma = 0; /* the paper's formality */
    REAL t1, t2, t3, t4;
    int code;
    REAL m = FABS(x1);
    if (m < FABS(x2)) {
        m = FABS(x2);
        if (m < FABS(x3)) m = FABS(x3);
        if (m < FABS(x4)) m = FABS(x4);
    } else {
        if (m < FABS(x3)) {
            m = FABS(x3);
            if (m < FABS(x4)) m = FABS(x4);
        } else {
            if (m >= FABS(x4)) {
                /* as in Scale3D: x2, x3 may be NaN when m = 0 */
                if (m == 0 && x2 == 0 && x3 == 0) {
                    y[0] = 0; y[1] = 0; y[2] = quat_zero ? 1 : 0; y[3] = 0;
                    *r = 0; *hout = 0;
                    return OR_CODE_ZERO;
                }
            } else {
                m = FABS(x4);
            }
        }
    }
    if (m >= TAU_MIN) {
        if (m <= TAU_MAX) {
            sigma = 1; t1 = x1; t2 = x2; t3 = x3; t4 = x4;
            code = OR_CODE_ONE;
        } else {
            sigma = INV_SIGMA_MAX;
            t1 = SIGMA_MAX * x1; t2 = SIGMA_MAX * x2;
            t3 = SIGMA_MAX * x3; t4 = SIGMA_MAX * x4;
            code = OR_CODE_SMAX;
        }
    } else {
        sigma = INV_SIGMA_MIN;
        t1 = SIGMA_MIN * x1; t2 = SIGMA_MIN * x2;
        t3 = SIGMA_MIN * x3; t4 = SIGMA_MIN * x4;
        code = OR_CODE_SMIN;
    }
    REAL rt = SQRT(t1 * t1 + t2 * t2 + t3 * t3 + t4 * t4);
    REAL h = 1 / rt;
    *r = sigma * rt;
    y[0] = h * t1;
    y[1] = h * t2;
    y[2] = h * t3;
    y[3] = h * t4;
    *hout = h;
    return code;
}

/* ---------------------------------------------------------------------- */
/* Canonical summation order CR(n) for n >= 5 (the paper only sums n <= 4
 * terms).  With S = OR_CR_SLOTS slots: slot j (j < min(n, S)) is the
 * left-to-right sum of the terms k = j, j + S, j + 2S, ...; then for
 * s = S/2, S/4, ..., 1 and each j < s, slot j <- slot j + slot (j + s) when
 * slot j + s holds a term (j + s < min(n, S)); absent slots are skipped, never
 * treated as +0.  The result is slot 0. */
static REAL SFX(cr_sum)(const REAL *term, int64_t n, REAL *slot)
{
    int64_t used = n < OR_CR_SLOTS ? n : OR_CR_SLOTS;
    for (int64_t j = 0; j < used; ++j) {
        REAL acc = term[j];
        for (int64_t k = j + OR_CR_SLOTS; k < n; k += OR_CR_SLOTS) acc = acc + term[k];
        slot[j] = acc;
    }
    for (int64_t s = OR_CR_SLOTS / 2; s >= 1; s /= 2)
        for (int64_t j = 0; j < s; ++j)
            if (j + s < used) slot[j] = slot[j] + slot[j + s];
    return slot[0];
}

/* Generic n (5 <= n <= 2^20): the steps of Algorithms 3-7 with m the largest
 * |x_k| over the components that are not NaN, the zero result iff every
 * component compares equal to zero, the constants TAU_MAX_N / SIGMA_MAX_N
 * (so that n tau_max^2 (1 + n u) <= omega for every n up to 2^20), and the
 * sum of squares in the order CR(n).  work holds 2n + OR_CR_SLOTS values. */
static int SFX(normalizeN)(const REAL *x, int64_t n, REAL *y, REAL *r, REAL *hout, REAL *work)
{
    REAL *t = work, *sq = work + n, *slot = work + 2 * n;
    int all_zero = 1;
    for (int64_t k = 0; k < n; ++k)
        if (!(x[k] == 0)) all_zero = 0;
    if (all_zero) {
        for (int64_t k = 0; k < n; ++k) y[k] = 0;
        *r = 0; *hout = 0;
        return OR_CODE_ZERO;
    }
    REAL m = 0;
    for (int64_t k = 0; k < n; ++k) {
        REAL a = FABS(x[k]);
        if (a > m) m = a;
    }
    REAL sigma, c;
    int code;
    if (m >= TAU_MIN) {
        if (m <= TAU_MAX_N) { sigma = 1; c = 1; code = OR_CODE_ONE; }
        else { sigma = INV_SIGMA_MAX_N; c = SIGMA_MAX_N; code = OR_CODE_SMAX; }
    } else {
        sigma = INV_SIGMA_MIN; c = SIGMA_MIN; code = OR_CODE_SMIN;
    }
    for (int64_t k = 0; k < n; ++k) t[k] = (code == OR_CODE_ONE) ? x[k] : c * x[k];
    for (int64_t k = 0; k < n; ++k) sq[k] = t[k] * t[k];
    REAL rt = SQRT(SFX(cr_sum)(sq, n, slot));
    REAL h = 1 / rt;
    *r = sigma * rt;
    for (int64_t k = 0; k < n; ++k) y[k] = h * t[k];
    *hout = h;
    return code;
}

/* One vector of any length.  quat_zero selects the [0,0,1,0] zero result of
 * Algorithm 7 for n = 4.  A zero-length vector has norm +0. */
static int SFX(normalize_one)(const REAL *x, int64_t n, REAL *y, REAL *r, REAL *h,
                              int quat_zero, REAL *work)
{
    switch (n) {
    case 0: *r = 0; *h = 0; return OR_CODE_ZERO;
    case 1: return SFX(normalize1)(x, y, r, h);
    case 2: return SFX(normalize2)(x, y, r, h);
    case 3: return SFX(normalize3)(x, y, r, h);
    case 4: return SFX(normalize4)(x, y, r, h, quat_zero);
    default: return SFX(normalizeN)(x, n, y, r, h, work);
    }
}

/* ---------------------------------------------------------------------- */
/* Backward pass of y = x / |x| (the paper has no derivative).  With the
 * forward's h = 1/r~ and factor c (x~ = c x, so 1/|x| = c h):
 *   dot = sum_k y_k g_k   (left to right for n <= 4, CR(n) otherwise)
 *   t_k = g_k - y_k * dot
 *   grad_k = (t_k * h) * c
 * and grad = +0 for a zero input vector. */
static void SFX(backward_one)(const REAL *y, const REAL *g, int64_t n, REAL h, int code,
                              REAL *grad, REAL *work)
{
    if (code == OR_CODE_ZERO) {
        for (int64_t k = 0; k < n; ++k) grad[k] = 0;
        return;
    }
    REAL c;
    if (code == OR_CODE_ONE) c = 1;
    else if (code == OR_CODE_SMIN) c = SIGMA_MIN;
    else c = (n <= 4) ? SIGMA_MAX : SIGMA_MAX_N;
    REAL dot;
    if (n <= 4) {
        dot = y[0] * g[0];
        for (int64_t k = 1; k < n; ++k) dot = dot + y[k] * g[k];
    } else {
        REAL *p = work, *slot = work + n;
        for (int64_t k = 0; k < n; ++k) p[k] = y[k] * g[k];
        dot = SFX(cr_sum)(p, n, slot);
    }
    for (int64_t k = 0; k < n; ++k) {
        REAL tk = g[k] - y[k] * dot;
        grad[k] = (tk * h) * c;
    }
}

/* ---------------------------------------------------------------------- */
/* Batch drivers with the library's layout: dim > 0 is a dense [count][dim]
 * batch, dim == 0 a ragged batch whose vector i is x[offsets[i] ..
 * offsets[i+1]).  norm, saved_h and saved_code may be NULL.  Returns 0, or
 * a nonzero value for bad arguments or a failed allocation. */
static int64_t SFX(max_len)(int64_t count, int32_t dim, const int64_t *offsets)
{
    if (dim > 0) return dim;
    int64_t mx = 0;
    for (int64_t i = 0; i < count; ++i) {
        int64_t n = offsets[i + 1] - offsets[i];
        if (n > mx) mx = n;
    }
    return mx;
}

int SFX(oracle_normalize)(const REAL *x, int64_t count, int32_t dim, const int64_t *offsets,
                          uint32_t flags, REAL *y, REAL *norm, REAL *saved_h, int8_t *saved_code)
{
    if (count < 0 || dim < 0 || (dim == 0 && offsets == NULL)) return 1;
    int64_t nmax = SFX(max_len)(count, dim, offsets);
    if (nmax > OR_MAX_LEN) return 2;
    REAL *work = (REAL *)malloc(sizeof(REAL) * (size_t)(2 * nmax + OR_CR_SLOTS));
    if (!work) return 3;
    int quat_zero = (dim == 4) && !(flags & OR_VECTOR_SEMANTICS);
    for (int64_t i = 0; i < count; ++i) {
        int64_t start = dim > 0 ? i * (int64_t)dim : offsets[i];
        int64_t n = dim > 0 ? dim : offsets[i + 1] - offsets[i];
        REAL r, h;
        int code = SFX(normalize_one)(x + start, n, y + start, &r, &h, quat_zero, work);
        if (norm) norm[i] = r;
        if (saved_h) saved_h[i] = h;
        if (saved_code) saved_code[i] = (int8_t)code;
    }
    free(work);
    return 0;
}

int SFX(oracle_backward)(const REAL *y, const REAL *g, const REAL *saved_h,
                         const int8_t *saved_code, int64_t count, int32_t dim,
                         const int64_t *offsets, REAL *grad)
{
    if (count < 0 || dim < 0 || (dim == 0 && offsets == NULL)) return 1;
    int64_t nmax = SFX(max_len)(count, dim, offsets);
    if (nmax > OR_MAX_LEN) return 2;
    REAL *work = (REAL *)malloc(sizeof(REAL) * (size_t)(nmax + OR_CR_SLOTS));
    if (!work) return 3;
    for (int64_t i = 0; i < count; ++i) {
        int64_t start = dim > 0 ? i * (int64_t)dim : offsets[i];
        int64_t n = dim > 0 ? dim : offsets[i + 1] - offsets[i];
        SFX(backward_one)(y + start, g + start, n, saved_h[i], saved_code[i], grad + start, work);
    }
    free(work);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Section 4: the rotation matrix of a quaternion (q1, q2, q3, q4) with scalar
 * part q4, from its normalization q^ by Algorithm 7 and the unit-norm form of
 * the matrix.  The printed unit-norm matrix has "2 q3^2" in its first and
 * "2 q2^2" in its last diagonal entry; the general matrix at |q| = 1 gives
 * 1 - 2(q2^2 + q3^2) and 1 - 2(q1^2 + q2^2), used here.  Each entry is
 * evaluated as written, row-major into R[9]. */
static void SFX(rotation_one)(const REAL *q, REAL *R, REAL *r)
{
    REAL u[4], h;
    SFX(normalize4)(q, u, r, &h, 1);
    REAL q1 = u[0], q2 = u[1], q3 = u[2], q4 = u[3];
    R[0] = 1 - 2 * (q2 * q2 + q3 * q3);
    R[1] = 2 * (q1 * q2 - q3 * q4);
    R[2] = 2 * (q1 * q3 + q2 * q4);
    R[3] = 2 * (q1 * q2 + q3 * q4);
    R[4] = 1 - 2 * (q1 * q1 + q3 * q3);
    R[5] = 2 * (q2 * q3 - q1 * q4);
    R[6] = 2 * (q1 * q3 - q2 * q4);
    R[7] = 2 * (q2 * q3 + q1 * q4);
    R[8] = 1 - 2 * (q1 * q1 + q2 * q2);
}

int SFX(oracle_rotation)(const REAL *q, int64_t count, REAL *R, REAL *norm)
{
    if (count < 0) return 1;
    for (int64_t i = 0; i < count; ++i) {
        REAL r;
        SFX(rotation_one)(q + 4 * i, R + 9 * i, &r);
        if (norm) norm[i] = r;
    }
    return 0;
}

/* ---------------------------------------------------------------------- */
/* The quotient algorithms the paper compares with (Section 1), for three
 * components.  They are not the method; the library builds them to measure
 * the paper's Table 3 ratio on the GPU.
 *
 * Algorithm 1 (robust quotient algorithm): m = max |x_k| (a NaN component
 * never compares greater), the zero case returns r = 0 and x unchanged;
 * otherwise t_k = x_k / m, r = m sqrt(t1 t1 + t2 t2 + t3 t3) and the
 * outputs are x_k / r.  Reading: the last step divides the input components
 * by r; the printed x_k <- x_k / r follows x_k <- x_k / m, which would return
 * x_k / (m r), not a unit vector. */
static void SFX(quotient1_3)(const REAL *x, REAL *y, REAL *r)
{
    REAL m = FABS(x[0]);
    if (FABS(x[1]) > m) m = FABS(x[1]);
    if (FABS(x[2]) > m) m = FABS(x[2]);
    if (m == 0) { *r = 0; y[0] = x[0]; y[1] = x[1]; y[2] = x[2]; return; }
    REAL t1 = x[0] / m, t2 = x[1] / m, t3 = x[2] / m;
    REAL rr = m * SQRT(t1 * t1 + t2 * t2 + t3 * t3);
    *r = rr;
    y[0] = x[0] / rr;
    y[1] = x[1] / rr;
    y[2] = x[2] / rr;
}

/* Lines 3-7 of Algorithm 2 with pivot xp (the component of largest
 * magnitude) and the other two components a, b in the roles of x1, x2. */
static void SFX(quotient2_pivot)(REAL xp, REAL a, REAL b, REAL *r, REAL *yp, REAL *ya, REAL *yb)
{
    REAL q1 = a / xp, q2 = b / xp;
    REAL h = SQRT(1 + q1 * q1 + q2 * q2);
    *r = FABS(xp) * h;
    REAL s = COPYSIGN((REAL)1, xp) / h;
    *ya = q1 * s;
    *yb = q2 * s;
    *yp = s;
}

/* Algorithm 2 (fast robust quotient algorithm), branch by branch: pivot x3
 * when |x1| > |x2| and |x3| > |x1|; pivot x1 (x1 and x3 exchange roles) when
 * |x1| > |x2| otherwise; pivot x3 when |x3| >= |x2| >= |x1|; pivot x2 (x2 and
 * x3 exchange roles) otherwise.  Reading: the zero return under "x3 = 0"
 * also requires x1 = 0, as the text promises NaN outputs for NaN inputs and
 * (NaN, 0, 0) reaches that test; with x1 = NaN the division gives NaN. */
static void SFX(quotient2_3)(const REAL *x, REAL *y, REAL *r)
{
    REAL x1 = x[0], x2 = x[1], x3 = x[2];
    if (FABS(x1) > FABS(x2)) {
        if (FABS(x3) > FABS(x1)) SFX(quotient2_pivot)(x3, x1, x2, r, &y[2], &y[0], &y[1]);
        else SFX(quotient2_pivot)(x1, x3, x2, r, &y[0], &y[2], &y[1]);
    } else {
        if (FABS(x3) >= FABS(x2)) {
            if (x3 == 0 && x1 == 0) { *r = 0; y[0] = 0; y[1] = 0; y[2] = 0; return; }
            SFX(quotient2_pivot)(x3, x1, x2, r, &y[2], &y[0], &y[1]);
        } else {
            SFX(quotient2_pivot)(x2, x1, x3, r, &y[1], &y[0], &y[2]);
        }
    }
}

/* Batch driver: x [count][3] -> y [count][3], r [count] (nullable);
 * alg = 1 or 2.  Returns 0, or 1 for bad arguments. */
int SFX(oracle_quotient3)(const REAL *x, int64_t count, int alg, REAL *y, REAL *norm)
{
    if (count < 0 || (alg != 1 && alg != 2)) return 1;
    for (int64_t i = 0; i < count; ++i) {
        REAL r;
        if (alg == 1) SFX(quotient1_3)(x + 3 * i, y + 3 * i, &r);
        else SFX(quotient2_3)(x + 3 * i, y + 3 * i, &r);
        if (norm) norm[i] = r;
    }
    return 0;
}

/* The naive sequence of the paper's Table 4 (no scaling): s = x1 x1 + ... +
 * xn xn (left to right), h = 1 / sqrt(s), y_k = h x_k; x [count][dim]. */
int SFX(oracle_naive)(const REAL *x, int64_t count, int32_t dim, REAL *y)
{
    if (count < 0 || dim < 1) return 1;
    for (int64_t i = 0; i < count; ++i) {
        const REAL *v = x + (int64_t)dim * i;
        REAL sum = v[0] * v[0];
        for (int32_t k = 1; k < dim; ++k) sum = sum + v[k] * v[k];
        REAL h = 1 / SQRT(sum);
        for (int32_t k = 0; k < dim; ++k) y[(int64_t)dim * i + k] = h * v[k];
    }
    return 0;
}
