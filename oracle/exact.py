"""Exact-arithmetic checks of a computed normalization against the paper's
error bounds (arXiv 1606.06508, Lemma 1 for n = 2, 3; Lemma 2 for
quaternions; Lemma 4 for the general form).

Every input is a binary32 or binary64 number, hence an exact dyadic rational.
The true norm r = sqrt(x_1^2 + ... + x_n^2) is irrational in general, so each
bound of the form |a - b/r| <= e is decided by squaring both sides with
their signs tracked, in exact rational arithmetic (``fractions``).  Nothing
here uses floating-point rounding, the oracle's C code, or the CUDA library.

TEST INFRASTRUCTURE: it pins the oracle (tests/) and measures the error of
computed results against the exact ones (the benchmark's accuracy report,
after its timed region); the library never imports it.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from fractions import Fraction as Fr

import numpy as np


@dataclass(frozen=True)
class Fmt:
    name: str
    u: Fr       # unit roundoff
    alpha: Fr   # smallest positive (subnormal) number
    nu: Fr      # smallest positive normal number
    omega: Fr   # largest finite number


F32 = Fmt("f32", Fr(1, 2 ** 24), Fr(1, 2 ** 149), Fr(1, 2 ** 126), Fr(2 ** 128 - 2 ** 104))
F64 = Fmt("f64", Fr(1, 2 ** 53), Fr(1, 2 ** 1074), Fr(1, 2 ** 1022), Fr(2 ** 1024 - 2 ** 971))


def fmt_of(dtype) -> Fmt:
    return F32 if np.dtype(dtype) == np.float32 else F64


def fr(v) -> Fr:
    return Fr(float(v))


def cr_depth(n: int, slots: int = 256) -> int:
    """Roundings on the longest path of a term through the order CR(n): one
    product, the sequential additions inside a slot, and one per tree level."""
    used = min(n, slots)
    levels = 0
    s = slots // 2
    while s >= 1:
        if s < used:
            levels += 1
        s //= 2
    return 1 + (math.ceil(n / slots) - 1) + levels


def rounds_in_sum(n: int) -> int:
    """k such that the computed sum of squares is (1 + theta) times the exact one
    with |theta| <= k u: n for the left-to-right sums of Algorithms 5-7
    (Lemma 4's proof), the depth of CR(n) otherwise."""
    return n if n <= 4 else cr_depth(n)


# Lemma 1: |sin phi| <= 1.001 u (n = 2, 3); Lemma 2: |q^_i q^_j - q_i q_j / r^2|
# <= (1.001 + 8.001 |q_i q_j| / r^2) u.
SIN_BOUND_U = Fr(1001, 1000)
PAIR_BOUND_U = (Fr(1001, 1000), Fr(8001, 1000))


def direction_bound(n: int, u: Fr) -> Fr:
    """Bound on ||x^ - x/r|| in units of u: (3.001 + n/2) for n <= 4 (Lemmas 1, 2,
    4); for n >= 5 the same proof with n u replaced by the rounding count k of
    the sum (and a k^2 u term for the first-order step)."""
    if n <= 4:
        return Fr(3001, 1000) + Fr(n, 2)
    k = rounds_in_sum(n)
    return Fr(3001, 1000) + Fr(k, 2) + k * k * u


def norm_bound(n: int, u: Fr) -> Fr:
    """Relative bound on |r^ - r| / r in units of u: (1 + n/2) (Lemmas 1, 2, 4)."""
    if n <= 4:
        return 1 + Fr(n, 2)
    k = rounds_in_sum(n)
    return 1 + Fr(k, 2) + k * k * u


def _le_sqrt_lhs(L: Fr, R: Fr, s: Fr) -> bool:
    """Decide L * sqrt(s) <= R exactly (s > 0)."""
    if L <= 0 and R >= 0:
        return True
    if L > 0 and R <= 0:
        return False
    if L > 0:
        return L * L * s <= R * R
    return L * L * s >= R * R  # L <= 0, R < 0


def _sqrt_approx(s: Fr, bits: int = 256) -> Fr:
    p, q = s.numerator, s.denominator
    return Fr(math.isqrt(p * q * (1 << (2 * bits))), q * (1 << bits))


@dataclass
class Result:
    n: int
    ok_direction: bool
    ok_norm: bool
    ok_finite: bool
    ok_sin: bool
    ok_pairs: bool
    err_direction_u: float   # ||x^ - x/r|| / u
    err_norm_u: float        # |r^ - r| / (r u)

    @property
    def ok(self) -> bool:
        return self.ok_direction and self.ok_norm and self.ok_finite and self.ok_sin and self.ok_pairs


def check(x, yhat, rhat, fmt: Fmt, quaternion: bool = False, dir_bound_u=None, norm_bound_u=None) -> Result:
    """Check one finite, nonzero input vector x and its computed (x^, r^).
    dir_bound_u / norm_bound_u replace the paper's bounds (Lemmas 1, 2, 4),
    for other algorithms checked with the same machinery."""
    n = len(x)
    xs = [fr(v) for v in x]
    if not all(math.isfinite(float(v)) for v in yhat):
        return Result(n, False, False, False, False, False, math.inf, math.inf)
    ys = [fr(v) for v in yhat]
    s = sum(v * v for v in xs)
    assert s > 0, "exact check needs a nonzero input"
    u = fmt.u
    A = sum(v * v for v in ys)
    P = sum(a * b for a, b in zip(ys, xs))
    # ||x^ - x/r||^2 = A - 2P/r + 1 <= (B u)^2  <=>  L <= 2P/r  <=>  L sqrt(s) <= 2P
    B = direction_bound(n, u) if dir_bound_u is None else Fr(dir_bound_u)
    L = A + 1 - (B * u) ** 2
    ok_dir = _le_sqrt_lhs(L, 2 * P, s)
    r_approx = _sqrt_approx(s)
    e2 = A - 2 * P / r_approx + 1
    err_dir = math.sqrt(max(float(e2), 0.0)) / float(u)

    # Lemma 1: |sin phi| <= 1.001 u for n = 2, 3:  s A - P^2 <= (1.001u)^2 s A
    ok_sin = True
    if n in (2, 3):
        ok_sin = s * A - P * P <= (SIN_BOUND_U * u) ** 2 * s * A

    # norm: finite and within (1 + n/2) r u (+ alpha/2 when 2r <= 3nu/2), claimed
    # when (1 + (1 + n/2) u) r <= omega
    rh = float(rhat)
    K = (norm_bound(n, u) if norm_bound_u is None else Fr(norm_bound_u)) * u
    finite_claim = (1 + K) ** 2 * s <= fmt.omega ** 2
    ok_fin = rh != 0.0 and (math.isfinite(rh) or not finite_claim)
    ok_norm = True
    err_norm = 0.0
    if finite_claim:
        if not math.isfinite(rh):
            ok_norm = False
            err_norm = math.inf
        else:
            R = fr(rh)
            e = fmt.alpha / 2 if 16 * s <= 9 * fmt.nu ** 2 else Fr(0)
            # R - r <= K r + e  <=>  R - e <= (1 + K) sqrt(s)
            up = _le_sqrt_lhs(-(1 + K), -(R - e), s)
            # r - R <= K r + e  <=>  (1 - K) sqrt(s) <= R + e
            lo = _le_sqrt_lhs(1 - K, R + e, s)
            ok_norm = up and lo
            err_norm = float(abs(R - r_approx) / r_approx) / float(u)

    # Lemma 2: |q^_i q^_j - q_i q_j / r^2| <= (1.001 + 8.001 |q_i q_j| / r^2) u
    ok_pairs = True
    if quaternion and n == 4:
        for i in range(4):
            for j in range(i, 4):
                exact = xs[i] * xs[j] / s
                if abs(ys[i] * ys[j] - exact) > (PAIR_BOUND_U[0] + PAIR_BOUND_U[1] * abs(exact)) * u:
                    ok_pairs = False
    return Result(n, ok_dir, ok_norm, ok_fin, ok_sin, ok_pairs, err_dir, err_norm)


def check_rows(args):
    """check() over rows (x, y^, r^), for a process pool: (fmt name, quaternion,
    xs, ys, rs) -> indices of the rows that fail, and the worst direction error
    in units of u.  Zero rows are skipped."""
    fmt_name, quaternion, xs, ys, rs = args
    fmt = F32 if fmt_name == "f32" else F64
    bad, worst = [], 0.0
    for i in range(len(xs)):
        if not np.any(xs[i] != 0):
            continue
        res = check(xs[i], ys[i], rs[i], fmt, quaternion=quaternion)
        if not res.ok:
            bad.append(i)
        worst = max(worst, res.err_direction_u)
    return bad, worst


def exact_gradient(x, g):
    """(g - x^ (x^ . g)) / r with x^ = x / r, as Fractions except for the one
    square root, carried to 256 bits.  Returns floats."""
    xs = [fr(v) for v in x]
    gs = [fr(v) for v in g]
    s = sum(v * v for v in xs)
    r = _sqrt_approx(s)
    dot_xg = sum(a * b for a, b in zip(xs, gs))
    # (g - x (x.g)/s) / r
    return [float((gk - xk * dot_xg / s) / r) for xk, gk in zip(xs, gs)]


def round_nearest_even(q: Fr, fmt: Fmt) -> float:
    """The binary32/binary64 number nearest to the rational q, ties to even,
    with gradual underflow (IEEE 754 roundTiesToEven), as a Python float.
    Written from the definition: scale q to an integer significand of p bits
    (or to the subnormal quantum alpha), round the integer, scale back."""
    if q == 0:
        return 0.0
    p = 24 if fmt is F32 else 53
    sign = -1.0 if q < 0 else 1.0
    a = abs(q)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fr(2) ** e > a:
        e -= 1
    # now 2^e <= a < 2^(e+1); quantum of the binade, not below alpha
    quantum = Fr(2) ** (e - (p - 1))
    if quantum < fmt.alpha:
        quantum = fmt.alpha
    m = a / quantum
    fl = m.numerator // m.denominator
    rem = m - fl
    if rem > Fr(1, 2) or (rem == Fr(1, 2) and fl % 2 == 1):
        fl += 1
    v = fl * quantum
    if v > fmt.omega:
        return sign * math.inf
    return sign * float(v)


def _ulp(v: Fr, fmt: Fmt) -> Fr:
    """Spacing of the binary32/binary64 numbers in the binade of |v| (alpha for
    v = 0 and for subnormal magnitudes)."""
    p = 24 if fmt is F32 else 53
    a = abs(v)
    if a == 0:
        return fmt.alpha
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fr(2) ** e > a:
        e -= 1
    q = Fr(2) ** (e - (p - 1))
    return q if q > fmt.alpha else fmt.alpha


def errors(x, yhat, rhat, fmt: Fmt) -> dict:
    """Measured errors of one computed (x^, r^) for a finite nonzero x, in
    units of u, with the exact norm carried to 256 bits (reporting, not a
    decision; check() decides the bounds exactly):
      direction_u  ||x^ - x/r||_2 / u         (Lemmas 1, 2, 4)
      norm_u       max(|r^ - r| - e, 0) / (r u), e = alpha/2 when 2r <= 3nu/2
                   (the absolute term Lemmas 1, 2, 4 allow for a subnormal
                   norm) and 0 otherwise; None if r^ is not finite
      sin_u        |sin phi| / u, phi the angle between x^ and x (Lemma 1)
      ulp          max_k |x^_k - x_k/r| / ulp(x_k/r)  (per component)."""
    xs = [fr(v) for v in x]
    if not all(math.isfinite(float(v)) for v in yhat):
        return {"direction_u": math.inf, "norm_u": math.inf, "sin_u": math.inf, "ulp": math.inf}
    ys = [fr(v) for v in yhat]
    s = sum(v * v for v in xs)
    r = _sqrt_approx(s)
    u = fmt.u
    A = sum(v * v for v in ys)
    P = sum(a * b for a, b in zip(ys, xs))
    e2 = A - 2 * P / r + 1
    direction = math.sqrt(max(float(e2), 0.0)) / float(u)
    sin2 = (s * A - P * P) / (s * A) if A > 0 else Fr(1)
    sin_u = math.sqrt(max(float(sin2), 0.0)) / float(u)
    rh = float(rhat)
    e = fmt.alpha / 2 if 16 * s <= 9 * fmt.nu ** 2 else Fr(0)
    norm_u = float(max(abs(fr(rh) - r) - e, Fr(0)) / r / u) if math.isfinite(rh) else None
    ulp = 0.0
    for xk, yk in zip(xs, ys):
        ex = xk / r
        ulp = max(ulp, float(abs(yk - ex) / _ulp(ex, fmt)))
    return {"direction_u": direction, "norm_u": norm_u, "sin_u": sin_u, "ulp": ulp}
