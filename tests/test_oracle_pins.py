"""Pins of the oracle to what the paper and mathematics fix (CPU only).

The oracle is the sequence of IEEE operations of Algorithms 3-7 of arXiv
1606.06508.  These tests tie it to things other than itself:
  - the constants of Table 2 against conditions (5)-(10) (condA-condF),
  - the thresholds the oracle actually applies, probed at tau_min / tau_max,
  - closed forms (Pythagorean tuples: exact norms, two roundings for x^),
  - invariants (sign flips, the first swap, power-of-two scaling),
  - special cases (NaN, zero, one nonzero component, infinities),
  - the error bounds of Lemmas 1, 2 and 4 decided in exact rational
    arithmetic on seeded samples, brute-force exponent sweeps and edge vectors,
  - the textbook sequence h = 1/sqrt(sum x^2), y = h x written independently
    with numpy scalars, for inputs that need no scaling.
"""
from fractions import Fraction as Fr
import math
import os

import numpy as np
import pytest

from oracle import exact
from gpu_util import full_grid_two_f32
from oracle.exact import F32, F64, fr
from paper_1606_06508_gb300 import synth

DT = {"f32": np.float32, "f64": np.float64}

TABLE2 = {  # Table 2: tau_min, sigma_min, tau_max, sigma_max
    "f32": (Fr(1, 2 ** 49), Fr(2 ** 100), Fr(2 ** 62), Fr(1, 2 ** 66)),
    "f64": (Fr(1, 2 ** 482), Fr(2 ** 592), Fr(2 ** 510), Fr(1, 2 ** 514)),
}
# constants for 5 <= n <= 2^20: tau_max = 2^floor((log2 omega - 21)/2), sigma_max = tau_max / 2^128 (f32)
GENERIC = {
    "f32": (Fr(1, 2 ** 49), Fr(2 ** 100), Fr(2 ** 53), Fr(1, 2 ** 75)),
    "f64": (Fr(1, 2 ** 482), Fr(2 ** 592), Fr(2 ** 501), Fr(1, 2 ** 523)),
}


def _is_pow2(q: Fr) -> bool:
    return q > 0 and q.numerator & (q.numerator - 1) == 0 and q.denominator & (q.denominator - 1) == 0


def _check_conditions(fmt, consts, nmax):
    tmin, smin, tmax, smax = consts
    u, a, nu, om = fmt.u, fmt.alpha, fmt.nu, fmt.omega
    # (5) condA: fl(nu^2) = 0 (nu^2 < alpha/2), u^2 >= 16 alpha, u <= 1e-6
    assert nu * nu < a / 2 and u * u >= 16 * a and u <= Fr(1, 10 ** 6)
    # (6) condB: powers of two
    assert _is_pow2(smin) and _is_pow2(smax)
    # (7) condC: u^2 tau_min^2 >= alpha and (n = 4: 8 tau_max^2 <= omega; generic: n (1+n u) tau_max^2 <= omega)
    assert u * u * tmin * tmin >= a
    assert max(8, nmax * (1 + nmax * u)) * tmax * tmax <= om
    # (8) condD: omega tau_min >= 1 and 3 nu tau_max <= 1
    assert om * tmin >= 1 and 3 * nu * tmax <= 1
    # (9) condE: x in (0, tau_min] => sigma_min x in [tau_min, tau_max] (x >= alpha)
    assert tmin <= smin * a and smin * tmin <= tmax
    # (10) condF: x in [tau_max, omega] => sigma_max x in [tau_min, tau_max]
    assert tmin <= smax * tmax and smax * om <= tmax


@pytest.mark.parametrize("f", ["f32", "f64"])
def test_table2_constants_satisfy_conditions(f):
    fmt = F32 if f == "f32" else F64
    _check_conditions(fmt, TABLE2[f], nmax=4)
    _check_conditions(fmt, GENERIC[f], nmax=1 << 20)
    tmin, smin, _, _ = TABLE2[f]
    assert smin * fmt.alpha == tmin  # the reading that keeps Table 2's tau_min


def test_eq4_formula_differs_from_table2():
    # Eq. (4) gives tau_min = 2^ceil(log2(alpha/u^2)/2): 2^-50 and 2^-484, while
    # Table 2 prints 2^-49 and 2^-482; tau_max agrees.  The oracle follows Table 2.
    for fmt, tmin_eq4, tmax_eq4, f in ((F32, -50, 62, "f32"), (F64, -484, 510, "f64")):
        lg = math.log2(fmt.alpha / fmt.u ** 2)
        assert math.ceil(lg / 2) == tmin_eq4
        assert math.floor((math.log2(fmt.omega) - 3) / 2) == tmax_eq4
        assert TABLE2[f][2] == Fr(2) ** tmax_eq4


def test_ieee_model(oracle_lib):
    assert oracle_lib.ieee_check()


# ---------------------------------------------------------------- thresholds
@pytest.mark.parametrize("f", ["f32", "f64"])
@pytest.mark.parametrize("n", [2, 3, 4, 5, 300])
def test_thresholds_applied(oracle_lib, f, n):
    """m = tau_min and m = tau_max need no scaling; the neighbours outside do."""
    dt = DT[f]
    tmin, _, tmax, _ = (TABLE2 if n <= 4 else GENERIC)[f]
    cases = [
        (float(tmin), 0), (float(np.nextafter(dt(float(tmin)), dt(0))), 1),
        (float(tmax), 0), (float(np.nextafter(dt(float(tmax)), dt(np.inf))), 2),
    ]
    for m, want in cases:
        x = np.zeros(n, dtype=dt)
        x[n // 2] = m
        x[0] = m / 4 if n // 2 != 0 else x[0]
        _, r, _, code = oracle_lib.normalize(x, dim=n, flags=1)
        assert code[0] == want, (f, n, m, code[0])


# ---------------------------------------------------------------- closed forms
PYTH = [(3, 4), (5, 12), (8, 15), (3, 4, 12), (2, 3, 6), (1, 2, 2), (4, 4, 7), (2, 6, 9), (6, 6, 7),
        (1, 4, 8), (8, 9, 12), (2, 4, 5, 6), (1, 2, 2, 4), (1, 1, 1, 1), (2, 2, 4, 5)]


@pytest.mark.parametrize("f", ["f32", "f64"])
def test_pythagorean_closed_form(oracle_lib, f):
    """Integer tuples with an integer norm R: the sum of squares and the square
    root are exact, so r^ = R and x^_k = RN(RN(1/R) x_k).  Holds after any
    scaling by 2^k that keeps every component and square normal."""
    fmt = F32 if f == "f32" else F64
    dt = DT[f]
    emax = 60 if f == "f32" else 500
    for tup in PYTH:
        R = math.isqrt(sum(v * v for v in tup))
        assert R * R == sum(v * v for v in tup)
        for k in (0, 7, -9, emax, -emax, 100 if f == "f32" else 1000, -100 if f == "f32" else -1000):
            x = np.array([v * 2.0 ** k for v in tup], dtype=dt)
            y, r, _, _ = oracle_lib.normalize(x, dim=len(tup), flags=1)
            assert float(r[0]) == R * 2.0 ** k
            h = exact.round_nearest_even(Fr(1, R), fmt)
            for xk, yk in zip(tup, y):
                assert float(yk) == exact.round_nearest_even(fr(h) * xk, fmt), (tup, k)


def test_values_show_the_method_is_not_correctly_rounded(oracle_lib):
    """Values that show the method is not correctly rounded (0 ulp is defined
    against the oracle, not against RN(x/r))."""
    y, *_ = oracle_lib.normalize(np.array([3.0, 4.0]), dim=2)
    assert y[0] == 0.6000000000000001 and y[1] == 0.8
    y, *_ = oracle_lib.normalize(np.array([49.0, 0.0, 0.0]), dim=3)
    assert y[0] == 0.9999999999999999
    y, *_ = oracle_lib.normalize(np.array([3, 4, 12], dtype=np.float32), dim=3)
    assert float(y[0]) == 0.23076924681663513 and float(y[2]) == 0.9230769872665405
    y, *_ = oracle_lib.normalize(np.array([2, 3, 6], dtype=np.float32), dim=3)
    assert float(y[1]) == 0.4285714626312256 and float(y[2]) == 0.8571429252624512


@pytest.mark.parametrize("f", ["f32", "f64"])
@pytest.mark.parametrize("n", [16, 64, 256, 289, 324, 529, 1024, 1089, 4096])
def test_generic_exact_integer_norm(oracle_lib, f, n):
    """n equal components 2^j: every partial sum is an exact small integer times
    2^2j in any order, so r^ = sqrt(n) 2^j exactly and no term may be dropped
    or counted twice by the order CR(n)."""
    dt = DT[f]
    for j in (0, 40, -40):
        x = np.full(n, 2.0 ** j, dtype=dt)
        y, r, _, code = oracle_lib.normalize(x, dim=n)
        assert float(r[0]) == math.isqrt(n) * 2.0 ** j
        assert np.all(y == y[0])
        # one component raised to 3 * 2^j adds exactly 8 * 4^j
        x[n - 1] = 3 * 2.0 ** j
        _, r, _, _ = oracle_lib.normalize(x, dim=n)
        want = math.sqrt(n + 8) * 2.0 ** j
        assert abs(float(r[0]) - want) <= 2 * want * float(F32.u if f == "f32" else F64.u)


# ---------------------------------------------------------------- invariants
@pytest.mark.parametrize("f", ["f32", "f64"])
@pytest.mark.parametrize("n", [2, 3, 4, 7, 256])
def test_sign_flip_and_swap(oracle_lib, f, n):
    dt = DT[f]
    x = synth.vectors_f32(2000, n, seed=11) if f == "f32" else synth.vectors_f64(2000, n, seed=11)
    y, r, h, c = oracle_lib.normalize(x.reshape(-1), dim=n)
    y = y.reshape(-1, n)
    for k in range(min(n, 4)):
        xf = x.copy()
        xf[:, k] = -xf[:, k]
        y2, r2, _, _ = oracle_lib.normalize(xf.reshape(-1), dim=n)
        y2 = y2.reshape(-1, n)
        exp = y.copy()
        exp[:, k] = -exp[:, k]
        assert np.array_equal(y2.view(np.uint8), exp.view(np.uint8))
        assert np.array_equal(r2, r)
    if n <= 4:  # the first addition commutes: swapping x1, x2 swaps the outputs exactly
        xs = x.copy()
        xs[:, [0, 1]] = xs[:, [1, 0]]
        y3, r3, _, _ = oracle_lib.normalize(xs.reshape(-1), dim=n)
        y3 = y3.reshape(-1, n)
        assert np.array_equal(y3[:, [1, 0]], y[:, [0, 1]]) and np.array_equal(r3, r)


@pytest.mark.parametrize("f", ["f32", "f64"])
@pytest.mark.parametrize("n", [2, 3, 4, 9])
def test_power_of_two_scaling(oracle_lib, f, n):
    """x -> 2^k x leaves x^ unchanged and scales r^ by 2^k when every component,
    every scaled component and every square stays normal in both evaluations
    (Lemma 3 and rndA)."""
    dt = DT[f]
    rng = np.random.default_rng(5)
    x = rng.uniform(0.5, 2.0, size=(3000, n)).astype(dt) * np.where(rng.integers(0, 2, (3000, n)) == 1, -1, 1)
    x = x.astype(dt)
    y, r, _, _ = oracle_lib.normalize(x.reshape(-1), dim=n)
    ks = (1, -3, 30, -30, 55, -45, 90, -110) if f == "f32" else (1, -3, 300, -300, 505, -470, 900, -1000)
    for k in ks:
        xs = np.ldexp(x, k).astype(dt)
        assert np.array_equal(np.ldexp(xs, -k), x)  # exact
        y2, r2, _, _ = oracle_lib.normalize(xs.reshape(-1), dim=n)
        assert np.array_equal(y2, y), k
        assert np.array_equal(r2, np.ldexp(r, k).astype(dt)), k


# ---------------------------------------------------------------- special cases
@pytest.mark.parametrize("f", ["f32", "f64"])
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 33])
def test_nan_propagates(oracle_lib, f, n):
    dt = DT[f]
    rng = np.random.default_rng(n)
    for k in range(n):
        for other in (0.0, 1.0, 1e30, 1e-30):
            x = np.full(n, other, dtype=dt) * rng.uniform(0.5, 1.5, n).astype(dt)
            x[k] = np.nan
            y, r, _, _ = oracle_lib.normalize(x, dim=n)
            assert np.all(np.isnan(y)) and np.isnan(r[0])
    x = rng.uniform(-1, 1, (50, n)).astype(dt)
    y, r, _, _ = oracle_lib.normalize(x.reshape(-1), dim=n)
    assert not np.any(np.isnan(y)) and not np.any(np.isnan(r))


@pytest.mark.parametrize("f", ["f32", "f64"])
@pytest.mark.parametrize("n", [1, 2, 3, 4, 6, 2000])
def test_zero_and_single_nonzero(oracle_lib, f, n):
    dt = DT[f]
    z = np.zeros(n, dtype=dt)
    z[::2] = -0.0
    y, r, h, c = oracle_lib.normalize(z, dim=n)
    if n == 4:
        assert y.tolist() == [0, 0, 1, 0]
    else:
        assert np.all(y == 0) and not np.any(np.signbit(y))
    assert r[0] == 0 and c[0] == 3
    y, r, _, _ = oracle_lib.normalize(z, dim=n, flags=1)
    assert np.all(y == 0)
    # one nonzero a: r^ = |a| exactly (fl(sqrt(fl(a^2))) = |a| without over/underflow)
    fi = np.finfo(dt)
    for a in (1.0, 49.0, -3.0, 1.5, float(fi.tiny), float(fi.smallest_subnormal) * 3, float(fi.max) / 3):
        x = np.zeros(n, dtype=dt)
        x[n - 1] = a
        y, r, _, _ = oracle_lib.normalize(x, dim=n, flags=1)
        assert float(r[0]) == abs(float(dt(a))), (n, a)
        assert abs(abs(float(y[n - 1])) - 1.0) <= 2 * float(fi.eps)
        assert np.sign(y[n - 1]) == np.sign(a)


@pytest.mark.parametrize("f", ["f32", "f64"])
def test_infinities_follow_the_operations(oracle_lib, f):
    """A component of +-inf: m = inf picks sigma_max, r~ = inf, h = 0, so x^ is NaN
    where x is infinite and +-0 elsewhere, and r^ = inf."""
    dt = DT[f]
    y, r, h, c = oracle_lib.normalize(np.array([np.inf, 1.0, -2.0], dtype=dt), dim=3)
    assert np.isnan(y[0]) and y[1] == 0 and y[2] == 0 and np.signbit(y[2]) and r[0] == np.inf
    assert c[0] == 2 and h[0] == 0


# ---------------------------------------------------------------- the textbook sequence
@pytest.mark.parametrize("f", ["f32", "f64"])
@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_unscaled_range_is_the_textbook_sequence(oracle_lib, f, n):
    """With tau_min <= m <= tau_max the method is h = 1/sqrt(x1^2 + ... + xn^2)
    (left to right), y = h x, r = sqrt(...), written here with numpy scalars."""
    dt = DT[f]
    rng = np.random.default_rng(100 + n)
    x = (rng.standard_normal((400, n)) * np.exp2(rng.integers(-40, 40, (400, 1)))).astype(dt)
    y, r, _, code = oracle_lib.normalize(x.reshape(-1), dim=n)
    assert np.all(code == 0)
    y = y.reshape(-1, n)
    one = dt(1)
    for i in range(x.shape[0]):
        acc = x[i, 0] * x[i, 0]
        for k in range(1, n):
            acc = dt(acc + dt(x[i, k] * x[i, k]))
        rt = np.sqrt(dt(acc))
        hh = dt(one / rt)
        assert r[i] == rt
        assert np.array_equal(y[i], (hh * x[i]).astype(dt))


# ---------------------------------------------------------------- error bounds (Lemmas 1, 2, 4)
def _bound_sweep(oracle_lib, x, n, f, quaternion=False, flags=0):
    fmt = F32 if f == "f32" else F64
    y, r, _, _ = oracle_lib.normalize(x.reshape(-1), dim=n, flags=flags)
    y = y.reshape(-1, n)
    worst = 0.0
    for i in range(x.shape[0]):
        if not np.any(x[i] != 0):
            continue
        res = exact.check(x[i], y[i], r[i], fmt, quaternion=quaternion)
        assert res.ok, (f, n, x[i].tolist(), y[i].tolist(), r[i], res)
        worst = max(worst, res.err_direction_u)
    return worst


def test_bounds_config0_vectors(oracle_lib):
    x = synth.vectors3_f64(4000, seed=0)
    _bound_sweep(oracle_lib, x, 3, "f64")


def test_bounds_edge_vectors(oracle_lib):
    _bound_sweep(oracle_lib, synth.edge_vectors_d3_f64(), 3, "f64")


def test_bounds_quaternions(oracle_lib):
    _bound_sweep(oracle_lib, synth.quaternions_f32(5000, seed=1), 4, "f32", quaternion=True)
    _bound_sweep(oracle_lib, synth.vectors_f64(3000, 4, seed=7), 4, "f64", quaternion=True)


@pytest.mark.parametrize("f", ["f32", "f64"])
def test_bounds_brute_force_two_components(oracle_lib, f):
    """n = 2 over an exponent grid covering the whole range (every 4th exponent
    pair), three mantissas and two sign patterns."""
    dt = DT[f]
    if f == "f32":
        es = list(range(-149, 128, 4)) + [127]
        mants = [1.0, 1.5, 2.0 - 2.0 ** -23]
    else:
        es = list(range(-1074, 1024, 31)) + [1023]
        mants = [1.0, 1.5, 2.0 - 2.0 ** -52]
    vals = []
    for e1 in es:
        for e2 in es:
            m1 = mants[(e1 + e2) % 3]
            m2 = mants[(e1 * 7 + e2) % 3]
            s2 = -1.0 if (e1 + e2) % 2 else 1.0
            vals.append((math.ldexp(m1, e1), s2 * math.ldexp(m2, e2)))
    x = np.array(vals, dtype=np.float64).astype(dt)
    _bound_sweep(oracle_lib, x, 2, f)


def _bounds_on_all_cores(oracle_lib, x, n, f, quaternion=False, chunk=20000):
    """The oracle's outputs for the rows of x within the paper's bounds, decided
    by exact.check on a spawn pool over the host cores; returns the worst
    direction error in units of u."""
    import multiprocessing as mp
    y, r, _, _ = oracle_lib.normalize(x.reshape(-1), dim=n)
    y = y.reshape(-1, n)
    chunks = [(a, min(a + chunk, x.shape[0])) for a in range(0, x.shape[0], chunk)]
    with mp.get_context("spawn").Pool(min(len(chunks), os.cpu_count() or 1)) as pool:
        res = pool.map(exact.check_rows, [(f, quaternion, x[a:b], y[a:b], r[a:b]) for a, b in chunks])
    bad = [a + i for (a, _), (failed, _) in zip(chunks, res) for i in failed]
    assert not bad, [x[i].tolist() for i in bad[:5]]
    return max(w for _, w in res)


def test_bounds_full_exponent_grid_two_components_f32(oracle_lib):
    """n = 2, binary32: the whole exponent grid (690,561 vectors) within the
    bounds of Lemma 1."""
    x = full_grid_two_f32()
    assert x.shape == (277 * 277 * 9, 2)
    assert _bounds_on_all_cores(oracle_lib, x, 2, "f32") <= 4.001


def test_bounds_whole_config0_and_sampled_quaternions(oracle_lib):
    """Every vector of the 65,600 x 3 binary64 case (Lemma 1), and 200,000
    binary32 quaternions of the headline recipe (Lemma 2, with the products
    q^_i q^_j)."""
    _bounds_on_all_cores(oracle_lib, synth.vectors3_f64(65536, seed=0), 3, "f64", chunk=5000)
    _bounds_on_all_cores(oracle_lib, synth.quaternions_f32(200000, seed=11), 4, "f32", quaternion=True,
                         chunk=5000)


@pytest.mark.parametrize("f", ["f32", "f64"])
@pytest.mark.parametrize("n", [3, 4])
def test_bounds_one_and_two_nonzero(oracle_lib, f, n):
    """Every placement of one or two nonzero components, each with 200 random
    exponents from the whole range (subnormals included) and random signs."""
    import itertools
    dt = DT[f]
    rng = np.random.default_rng(31 + n)
    emin, emax = (-149, 127) if f == "f32" else (-1074, 1023)
    xs = []
    for size in (1, 2):
        for pos in itertools.combinations(range(n), size):
            for _ in range(200):
                x = np.zeros(n)
                sign = np.where(rng.integers(0, 2, size) == 1, -1.0, 1.0)
                x[list(pos)] = sign * np.ldexp(rng.uniform(1, 2, size), rng.integers(emin, emax + 1, size))
                xs.append(x)
    _bound_sweep(oracle_lib, np.array(xs).astype(dt), n, f, flags=1)


@pytest.mark.parametrize("f", ["f32", "f64"])
@pytest.mark.parametrize("n", [5, 37, 256, 1500])
def test_bounds_generic_rows(oracle_lib, f, n):
    dt = DT[f]
    cnt = {5: 300, 37: 120, 256: 24, 1500: 6}[n]
    x = synth.rows(cnt, n, dt, seed=2)
    _bound_sweep(oracle_lib, x, n, f)
    xw = synth.vectors_f32(cnt, n, seed=3) if f == "f32" else synth.vectors_f64(cnt, n, seed=3)
    _bound_sweep(oracle_lib, xw, n, f)


# ---------------------------------------------------------------- batch layouts
@pytest.mark.parametrize("f", ["f32", "f64"])
def test_ragged_equals_fixed(oracle_lib, f):
    """A ragged vector of length n gives the bits of a dense batch of dimension n
    (vector zero rule for n = 4); a zero-length vector has norm +0."""
    dt = DT[f]
    lengths = np.array([0, 1, 2, 3, 4, 5, 8, 31, 300, 0, 4, 1025, 2], dtype=np.int64)
    off = synth.offsets_from_lengths(lengths)
    x = synth.ragged_values(lengths, dt, seed=9)
    x[off[10]:off[11]] = 0  # a zero vector of length 4
    y, r, h, c = oracle_lib.normalize(x, dim=0, offsets=off)
    for i, n in enumerate(lengths):
        if n == 0:
            assert r[i] == 0
            continue
        yi, ri, hi, ci = oracle_lib.normalize(x[off[i]:off[i + 1]], dim=int(n), flags=1)
        assert np.array_equal(y[off[i]:off[i + 1]].view(np.uint8), yi.view(np.uint8))
        assert r[i] == ri[0] and h[i] == hi[0] and c[i] == ci[0]


# ---------------------------------------------------------------- backward
@pytest.mark.parametrize("f", ["f32", "f64"])
@pytest.mark.parametrize("n", [2, 3, 4, 6, 100])
def test_backward_against_exact_gradient(oracle_lib, f, n):
    dt = DT[f]
    fmt = F32 if f == "f32" else F64
    cnt = 300 if n < 100 else 40
    x = synth.rows(cnt, n, dt, seed=21, smax=60 if f == "f32" else 600)
    g = synth.normal_like((cnt, n), dt, seed=22)
    y, r, h, c = oracle_lib.normalize(x.reshape(-1), dim=n, flags=1)
    grad = oracle_lib.backward(y, g.reshape(-1), h, c, dim=n).reshape(-1, n)
    k = exact.rounds_in_sum(n)
    C = 2 * (float(exact.direction_bound(n, fmt.u)) + k + 4)
    for i in range(cnt):
        ex = exact.exact_gradient(x[i], g[i])
        scale = float(np.linalg.norm(g[i].astype(np.float64))) / float(r[i])
        err = max(abs(float(a) - b) for a, b in zip(grad[i], ex))
        assert err <= C * float(fmt.u) * scale, (i, err / (float(fmt.u) * scale))


@pytest.mark.parametrize("n", [3, 4, 50])
def test_backward_against_central_differences(oracle_lib, n):
    """FP64 central differences of the oracle's forward, step 1e-6 |x|."""
    cnt = 64
    x = synth.rows(cnt, n, np.float64, seed=41, smax=300)
    g = synth.normal_like((cnt, n), np.float64, seed=42)
    y, r, h, c = oracle_lib.normalize(x.reshape(-1), dim=n, flags=1)
    grad = oracle_lib.backward(y, g.reshape(-1), h, c, dim=n).reshape(-1, n)
    for i in range(cnt):
        step = 1e-6 * float(r[i])
        fd = np.empty(n)
        for k in range(n):
            xp = x[i].copy()
            xm = x[i].copy()
            xp[k] += step
            xm[k] -= step
            yp = oracle_lib.normalize(xp, dim=n, flags=1)[0]
            ym = oracle_lib.normalize(xm, dim=n, flags=1)[0]
            fd[k] = np.dot(g[i], (yp - ym)) / (2 * step)
        scale = np.linalg.norm(g[i]) / float(r[i])
        assert np.max(np.abs(fd - grad[i])) <= 1e-7 * scale


def test_backward_zero_vector(oracle_lib):
    for n, flags in ((3, 0), (4, 0), (4, 1), (9, 0)):
        x = np.zeros(n)
        y, r, h, c = oracle_lib.normalize(x, dim=n, flags=flags)
        grad = oracle_lib.backward(y, np.ones(n), h, c, dim=n)
        assert np.all(grad == 0) and not np.any(np.signbit(grad))


# ---------------------------------------------------------------- rotation matrix (Section 4)
@pytest.mark.parametrize("f", ["f32", "f64"])
def test_rotation_against_exact_matrix(oracle_lib, f):
    """R(q^) against the exact R(q) = (general matrix) / |q|^2 in rational
    arithmetic.  Lemma 2 bounds |q^_i q^_j - q_i q_j / r^2| by
    (1.001 + 8.001 |q_i q_j| / r^2) u; each entry adds at most three more
    roundings of values <= 2, so every entry is within 30 u."""
    fmt = F32 if f == "f32" else F64
    dt = DT[f]
    q = synth.quaternions_f32(1500, seed=12).astype(dt) if f == "f32" else synth.vectors_f64(1500, 4, seed=12)
    R, r = oracle_lib.rotation(q)
    u = fmt.u
    for i in range(q.shape[0]):
        a, b, c, d = (fr(v) for v in q[i])
        s = a * a + b * b + c * c + d * d
        if s == 0:
            continue
        ex = [[a * a + d * d - b * b - c * c, 2 * (a * b - c * d), 2 * (a * c + b * d)],
              [2 * (a * b + c * d), b * b + d * d - a * a - c * c, 2 * (b * c - a * d)],
              [2 * (a * c - b * d), 2 * (b * c + a * d), c * c + d * d - a * a - b * b]]
        for j in range(3):
            for k in range(3):
                assert abs(fr(R[i, j, k]) - ex[j][k] / s) <= 30 * u, (i, j, k)


def test_rotation_special_cases(oracle_lib):
    R, r = oracle_lib.rotation(np.zeros((1, 4)))
    assert R[0].tolist() == [[-1, 0, 0], [0, -1, 0], [0, 0, 1]] and r[0] == 0  # q^ = (0, 0, 1, 0)
    R, _ = oracle_lib.rotation(np.array([[0.0, 0.0, 0.0, 5.0]]))
    assert R[0].tolist() == [[1, 0, 0], [0, 1, 0], [0, 0, 1]]
    R, _ = oracle_lib.rotation(np.array([[2.0 ** -1000, 0.0, 0.0, 0.0]]))  # tiny: scaled; half turn about axis 1
    assert R[0].tolist() == [[1, 0, 0], [0, -1, 0], [0, 0, -1]]
