"""Pins of the oracle's quotient algorithms (Algorithms 1 and 2, Section 1)
and of the naive sequence (Table 4), none of which reuses the oracle's code:
exact-arithmetic error bounds derived for each algorithm's operation count,
special cases with known results, and the readings taken for the printed
algorithms (the last step of Algorithm 1, the zero test of Algorithm 2).

Bounds (u the unit roundoff; derived from the operation count of each
algorithm, as the paper does for its own in Lemma 1):
  Algorithm 2: q_k = x_k / x_p (1 rounding), q_k^2 (3), the sum (2 more), the
  square root (h within 3.5u), r = |x_p| h (4.5u), s = sign / h (4.5u),
  y_k = q_k s (6.5u): ||y - x/r|| <= 8u and |r^ - r| <= 6u r.
  Algorithm 1: t_k = x_k / m (1), t_k^2 (3), the sum (5), the square root
  (3.5u), r = m sqrt (4.5u), y_k = x_k / r (5.5u): the same 8u and 6u, for
  norms far from the subnormal range (r is formed, then divided into x).
"""
import math

import numpy as np
import pytest

import oracle
from oracle.exact import F32, F64, check

FMT = {np.float32: F32, np.float64: F64}


def _wide3(rng, count, dt):
    """Components sign x U[1,2) x 2^e with a per-vector base exponent and a
    spread, so the vectors have components of very different sizes."""
    if dt == np.float32:
        lo, hi, spread = -100, 90, 30
    else:
        lo, hi, spread = -900, 800, 200
    base = rng.integers(lo, hi, size=(count, 1))
    e = base + rng.integers(-spread, spread + 1, size=(count, 3))
    m = rng.uniform(1.0, 2.0, size=(count, 3)) * rng.choice([-1.0, 1.0], size=(count, 3))
    return np.ldexp(m, e).astype(dt)


@pytest.mark.parametrize("dt", [np.float32, np.float64])
@pytest.mark.parametrize("alg", [1, 2])
def test_quotient_exact_bounds(dt, alg):
    rng = np.random.default_rng(7 + alg)
    x = _wide3(rng, 1500, dt)
    x[:40] = rng.standard_normal((40, 3)).astype(dt)
    x[40:50, 1] = 0
    y, r = oracle.quotient3(x, alg)
    fmt = FMT[dt]
    nbad = 0
    for i in range(len(x)):
        res = check(x[i], y[i], r[i], fmt, dir_bound_u=8, norm_bound_u=6)
        nbad += not (res.ok_direction and res.ok_norm)
    assert nbad == 0


@pytest.mark.parametrize("dt", [np.float32, np.float64])
@pytest.mark.parametrize("alg", [1, 2])
def test_quotient_special_cases(dt, alg):
    z = np.zeros((1, 3), dt)
    y, r = oracle.quotient3(z, alg)
    assert r[0] == 0 and not np.any(y)
    for pos in range(3):
        for a in (dt(-5), dt(0.75), dt(np.finfo(dt).max), dt(np.finfo(dt).tiny)):
            x = np.zeros((1, 3), dt)
            x[0, pos] = a
            y, r = oracle.quotient3(x, alg)
            assert r[0] == abs(a)
            want = np.zeros(3, dt)
            want[pos] = math.copysign(1.0, float(a))
            assert np.array_equal(np.abs(y[0]), np.abs(want)) and y[0, pos] == want[pos]


@pytest.mark.parametrize("dt", [np.float32, np.float64])
def test_quotient2_nan_propagates(dt):
    """The text promises NaN outputs for NaN inputs; with the zero test read
    as x1 = x3 = 0 that holds in every position, (NaN, 0, 0) included."""
    for pos in range(3):
        for others in ((0, 0), (1, 2), (0, 3)):
            x = np.array([[others[0], others[1], 0]], dt)
            x = np.insert(x[:, :2], pos, np.nan, axis=1)
            y, r = oracle.quotient3(x, 2)
            assert np.all(np.isnan(y)) and np.isnan(r[0]), (pos, others)


def test_quotient1_last_step_divides_the_input():
    """Reading of Algorithm 1's last line: the outputs are x_k / r with the
    input x_k; the scaled t_k / r would be x_k / (m r)."""
    x = np.array([[3.0, 4.0, 12.0], [2.0 ** 40, 0.0, 2.0 ** 40]])
    y, r = oracle.quotient3(x, 1)
    assert r[0] == 13.0 and abs(np.linalg.norm(y[0]) - 1) < 1e-15
    assert abs(np.linalg.norm(y[1]) - 1) < 1e-15


@pytest.mark.parametrize("dt", [np.float32, np.float64])
def test_naive_sequence(dt):
    """The naive sequence overflows and underflows where the scaling does not,
    and equals the scaling algorithm's result when no scaling is needed
    (c = 1 with tau_min <= m <= tau_max: the same operations)."""
    rng = np.random.default_rng(3)
    x = rng.standard_normal((500, 3)).astype(dt)
    y = oracle.naive(x, 3)
    ys, _, _, codes = oracle.normalize(x.reshape(-1), dim=3)
    assert np.all(codes == 0)
    assert np.array_equal(y.view(np.uint8), ys.reshape(500, 3).view(np.uint8))
    big = np.array([[np.finfo(dt).max, np.finfo(dt).max, 0]], dt)
    assert np.all(oracle.naive(big, 3)[0, :2] == 0)  # 1/inf = 0
    tiny = np.array([[np.finfo(dt).smallest_subnormal, 0, 0]], dt)
    assert np.isinf(oracle.naive(tiny, 3)[0, 0])     # the square underflows to 0
