"""Seeded synthetic inputs shaped like the workloads of arXiv 1606.06508.

The paper times its algorithms on unspecified inputs (Appendix A) and uses no
dataset, so these generators stand in for its workloads: 2-, 3- and
4-component vectors and quaternions, long rows and ragged batches, with
exponents spread wide enough that an unscaled sum of squares would overflow
or underflow.

This module draws random numbers and nothing else: it holds none of the
method's arithmetic.  It serves both sides of every parity test (the CUDA
library and the oracle) and the benchmark.  Each generator has a numpy
backend (host arrays, for sizes the oracle handles) and a torch backend
(device tensors, for full-size runs); the two draw different streams with the
same distribution.
"""
from __future__ import annotations

import math

import numpy as np

# --------------------------------------------------------------------------
# 64 fixed three-component binary64 vectors: zeros, one nonzero component,
# Pythagorean triples (exact norms) with sign flips, permutations and power of
# two scalings, near-overflow and subnormal magnitudes, and the scaling
# thresholds of Table 2 (2^-482 and 2^510) and their neighbours.
_OMEGA = float(np.finfo(np.float64).max)
_TINY = 2.0 ** -1074


def edge_vectors_d3_f64() -> np.ndarray:
    p = 2.0 ** 1000
    q = 2.0 ** -1060
    just_below_2m482 = float(np.nextafter(2.0 ** -482, 0.0))
    just_above_2p510 = float(np.nextafter(2.0 ** 510, np.inf))
    rows = [
        (0.0, 0.0, 0.0), (-0.0, 0.0, 0.0), (0.0, -0.0, -0.0), (-0.0, -0.0, -0.0),
        (1.0, 0.0, 0.0), (0.0, 49.0, 0.0), (0.0, 0.0, -3.0), (1.5 * p, 0.0, 0.0),
        (0.0, q, 0.0), (0.0, 0.0, -_TINY),
        (3.0, 4.0, 12.0), (2.0, 3.0, 6.0), (1.0, 2.0, 2.0), (4.0, 4.0, 7.0),
        (2.0, 6.0, 9.0), (6.0, 6.0, 7.0), (1.0, 4.0, 8.0), (8.0, 9.0, 12.0),
        (-3.0, 4.0, -12.0), (12.0, 3.0, 4.0), (6.0, -2.0, 3.0), (-2.0, -1.0, -2.0),
        (7.0, 4.0, 4.0), (9.0, 6.0, 2.0),
        (3 * p, 4 * p, 12 * p), (2 * p, 3 * p, 6 * p), (1 * p, 2 * p, 2 * p), (8 * p, 9 * p, 12 * p),
        (3 * q, 4 * q, 12 * q), (2 * q, 3 * q, 6 * q), (1 * q, 2 * q, 2 * q), (4 * q, 4 * q, 7 * q),
        (1.9 * 2.0 ** 1023, 1.9 * 2.0 ** 1023, 2.0 ** 1023), (2.0 ** 1023, 2.0 ** 1023, 0.0),
        (_OMEGA, 0.0, 0.0), (_OMEGA, _OMEGA, _OMEGA), (-_OMEGA, _OMEGA, -_OMEGA),
        (2.0 ** 1022, 2.0 ** 1022, 2.0 ** 1022), (1.5 * 2.0 ** 1023, _TINY, 0.0),
        (2.0 ** 511, 2.0 ** 511, 2.0 ** 511),
        (2.0 ** 510, 0.0, 0.0), (just_above_2p510, 1.0, 1.0), (2.0 ** -482, 0.0, 0.0),
        (just_below_2m482, 0.0, 0.0), (2.0 ** -482, 2.0 ** -482, 2.0 ** -482), (2.0 ** -483, 1e-300, 0.0),
        (p, q, 1.0), (q, p, -_TINY), (1.0, 2.0 ** -600, 2.0 ** -600), (2.0 ** -1000, q, _TINY),
        (_TINY, _TINY, _TINY), (_TINY, 0.0, -_TINY), (1e-320, 1e-320, 1e-320), (1.0, 1e-200, 1e-200),
        (1.0, 1.0, 1.0), (1.0, 1e-8, 0.0), (0.6, 0.8, 0.0), (1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0),
        (-1.0, -1.0, -1.0), (1e-10, 1e-10, 1e-10), (1e10, 1e10, 1e10), (1.0000000000000002, 0.0, 0.0),
        (0.5, 0.5, 0.7071067811865476), (2.0 ** -30, 2.0 ** 30, 1.0),
    ]
    a = np.array(rows, dtype=np.float64)
    assert a.shape == (64, 3)
    return a


# --------------------------------------------------------------------------
# numpy backend
def _np_sign_mant_exp(rng, size, emin, emax, mant_bits):
    """random sign x mantissa uniform on [1, 2) with mant_bits random bits x 2^e,
    e a uniform integer in [emin, emax], formed exactly in binary64."""
    sign = np.where(rng.integers(0, 2, size=size) == 1, -1.0, 1.0)
    mant = 1.0 + rng.integers(0, 1 << mant_bits, size=size, dtype=np.int64).astype(np.float64) \
        * (2.0 ** -mant_bits)
    e = rng.integers(emin, emax + 1, size=size)
    return np.ldexp(sign * mant, e)


def vectors3_f64(count: int = 65536, seed: int = 0, edges: bool = True) -> np.ndarray:
    """count x 3 binary64 vectors, each component random sign x U[1,2) (52 random
    fraction bits) x 2^e with e uniform in [-30, 30]; then the 64 edge vectors."""
    rng = np.random.default_rng(seed)
    x = _np_sign_mant_exp(rng, (count, 3), -30, 30, 52)
    if edges:
        x = np.concatenate([x, edge_vectors_d3_f64()], axis=0)
    return np.ascontiguousarray(x)


def quaternions_f32(count: int, seed: int = 1) -> np.ndarray:
    """count x 4 binary32 quaternions.  Per component, with probability 1/2:
    random sign x U[1,2) (23 random bits) x 2^e, e uniform in [-149, 127],
    rounded to binary32 (e < -126 gives subnormals); otherwise N(0,1) rounded
    to binary32."""
    rng = np.random.default_rng(seed)
    wide = _np_sign_mant_exp(rng, (count, 4), -149, 127, 23).astype(np.float32)
    normal = rng.standard_normal((count, 4)).astype(np.float32)
    pick = rng.integers(0, 2, size=(count, 4)) == 1
    return np.ascontiguousarray(np.where(pick, wide, normal))


def quaternions_f64(count: int, seed: int = 5) -> np.ndarray:
    """count x 4 binary64 quaternions, each component drawn like those of
    :func:`vectors3_f64`: random sign x U[1,2) (52 random fraction bits) x 2^e,
    e uniform in [-30, 30]."""
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(_np_sign_mant_exp(rng, (count, 4), -30, 30, 52))


def vectors_f32(count: int, dim: int, seed: int) -> np.ndarray:
    """count x dim binary32 vectors drawn like the quaternion components."""
    rng = np.random.default_rng(seed)
    wide = _np_sign_mant_exp(rng, (count, dim), -149, 127, 23).astype(np.float32)
    normal = rng.standard_normal((count, dim)).astype(np.float32)
    pick = rng.integers(0, 2, size=(count, dim)) == 1
    return np.ascontiguousarray(np.where(pick, wide, normal))


def vectors_f64(count: int, dim: int, seed: int) -> np.ndarray:
    """count x dim binary64 vectors: half the components random sign x U[1,2) x
    2^e with e uniform over the whole binary64 range (subnormals included),
    half N(0,1)."""
    rng = np.random.default_rng(seed)
    wide = _np_sign_mant_exp(rng, (count, dim), -1074, 1023, 52)
    normal = rng.standard_normal((count, dim))
    pick = rng.integers(0, 2, size=(count, dim)) == 1
    return np.ascontiguousarray(np.where(pick, wide, normal))


def rows(count: int, dim: int, dtype, seed: int = 2, smax: int | None = None) -> np.ndarray:
    """count x dim rows, x = N(0,1) x 2^s with one s per row, uniform in
    [-smax, smax] (defaults: 120 for binary32, 1000 for binary64)."""
    dtype = np.dtype(dtype)
    if smax is None:
        smax = 120 if dtype == np.float32 else 1000
    rng = np.random.default_rng(seed)
    s = rng.integers(-smax, smax + 1, size=(count, 1))
    z = rng.standard_normal((count, dim)).astype(dtype)
    return np.ascontiguousarray(np.ldexp(z, s.astype(np.int32)).astype(dtype))


def ragged_lengths(count: int, seed: int = 3, kind: str = "mixture", nmax: int = 4096) -> np.ndarray:
    """Vector lengths.  'mixture': with probability 0.4 uniform in {2, 3, 4},
    otherwise floor(exp(U(ln 5, ln(nmax + 1)))); 'loguniform':
    floor(exp(U(ln 2, ln(nmax + 1))))."""
    rng = np.random.default_rng(seed)
    if kind == "mixture":
        short = rng.integers(2, 5, size=count)
        long_ = np.floor(np.exp(rng.uniform(math.log(5), math.log(nmax + 1), size=count)))
        n = np.where(rng.uniform(size=count) < 0.4, short, long_)
    elif kind == "loguniform":
        n = np.floor(np.exp(rng.uniform(math.log(2), math.log(nmax + 1), size=count)))
    else:
        raise ValueError(kind)
    return np.clip(n, 1, nmax).astype(np.int64)


def offsets_from_lengths(lengths) -> np.ndarray:
    off = np.zeros(len(lengths) + 1, dtype=np.int64)
    np.cumsum(lengths, out=off[1:])
    return off


def ragged_values(lengths, dtype, seed: int = 3, smax: int = 100) -> np.ndarray:
    """Packed components of a ragged batch: N(0,1) x 2^s, one s per vector,
    uniform in [-smax, smax]."""
    dtype = np.dtype(dtype)
    lengths = np.asarray(lengths, dtype=np.int64)
    rng = np.random.default_rng(seed + 1000)
    s = rng.integers(-smax, smax + 1, size=lengths.size).astype(np.int32)
    z = rng.standard_normal(int(lengths.sum())).astype(dtype)
    return np.ascontiguousarray(np.ldexp(z, np.repeat(s, lengths)).astype(dtype))


def normal_like(shape, dtype, seed: int = 4) -> np.ndarray:
    """i.i.d. N(0,1) values (upstream gradients)."""
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(rng.standard_normal(shape).astype(np.dtype(dtype)))


# --------------------------------------------------------------------------
# torch backend (device tensors for full-size runs)
def _torch():
    import torch
    return torch


def _tgen(seed, device):
    torch = _torch()
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    return g


def _t_sign_mant_exp(g, shape, emin, emax, mant_bits, device):
    torch = _torch()
    sign = torch.randint(0, 2, shape, generator=g, device=device, dtype=torch.int32) * 2 - 1
    frac = torch.randint(0, 1 << mant_bits, shape, generator=g, device=device, dtype=torch.int64)
    mant = 1.0 + frac.to(torch.float64) * (2.0 ** -mant_bits)
    e = torch.randint(emin, emax + 1, shape, generator=g, device=device, dtype=torch.int32)
    return torch.ldexp(sign.to(torch.float64) * mant, e.to(torch.float64))


def quaternions_f32_torch(count: int, seed: int = 1, device="cuda"):
    """Device version of :func:`quaternions_f32` (same distribution, chunked)."""
    torch = _torch()
    g = _tgen(seed, device)
    out = torch.empty((count, 4), dtype=torch.float32, device=device)
    chunk = 1 << 22
    for a in range(0, count, chunk):
        b = min(count, a + chunk)
        shp = (b - a, 4)
        wide = _t_sign_mant_exp(g, shp, -149, 127, 23, device).to(torch.float32)
        normal = torch.randn(shp, generator=g, device=device, dtype=torch.float32)
        pick = torch.randint(0, 2, shp, generator=g, device=device, dtype=torch.int32) == 1
        out[a:b] = torch.where(pick, wide, normal)
    return out


def quaternions_f64_torch(count: int, seed: int = 5, device="cuda"):
    """Device version of :func:`quaternions_f64` (same distribution, chunked)."""
    torch = _torch()
    g = _tgen(seed, device)
    out = torch.empty((count, 4), dtype=torch.float64, device=device)
    chunk = 1 << 22
    for a in range(0, count, chunk):
        b = min(count, a + chunk)
        out[a:b] = _t_sign_mant_exp(g, (b - a, 4), -30, 30, 52, device)
    return out


def rows_torch(count: int, dim: int, dtype, seed: int = 2, smax: int | None = None, device="cuda"):
    """Device version of :func:`rows`."""
    torch = _torch()
    if smax is None:
        smax = 120 if dtype == torch.float32 else 1000
    g = _tgen(seed, device)
    s = torch.randint(-smax, smax + 1, (count, 1), generator=g, device=device, dtype=torch.int32)
    out = torch.randn((count, dim), generator=g, device=device, dtype=dtype)
    return torch.ldexp(out, s.to(dtype))


def ragged_lengths_torch(count: int, seed: int = 3, kind: str = "mixture", nmax: int = 4096, device="cuda"):
    """Device version of :func:`ragged_lengths`."""
    torch = _torch()
    g = _tgen(seed, device)
    if kind == "mixture":
        short = torch.randint(2, 5, (count,), generator=g, device=device, dtype=torch.int64)
        u = torch.rand((count,), generator=g, device=device, dtype=torch.float64)
        long_ = torch.floor(torch.exp(math.log(5) + u * (math.log(nmax + 1) - math.log(5))))
        pick = torch.rand((count,), generator=g, device=device, dtype=torch.float64) < 0.4
        n = torch.where(pick, short.to(torch.float64), long_)
    elif kind == "loguniform":
        u = torch.rand((count,), generator=g, device=device, dtype=torch.float64)
        n = torch.floor(torch.exp(math.log(2) + u * (math.log(nmax + 1) - math.log(2))))
    else:
        raise ValueError(kind)
    return torch.clamp(n, 1, nmax).to(torch.int64)


def offsets_from_lengths_torch(lengths):
    torch = _torch()
    off = torch.zeros(lengths.numel() + 1, dtype=torch.int64, device=lengths.device)
    torch.cumsum(lengths, 0, out=off[1:])
    return off


def ragged_values_torch(lengths, dtype, seed: int = 3, smax: int = 100):
    """Device version of :func:`ragged_values`."""
    torch = _torch()
    device = lengths.device
    g = _tgen(seed + 1000, device)
    s = torch.randint(-smax, smax + 1, (lengths.numel(),), generator=g, device=device, dtype=torch.int16)
    total = int(lengths.sum().item())
    z = torch.randn(total, generator=g, device=device, dtype=dtype)
    e = torch.repeat_interleave(s, lengths, output_size=total)
    # ldexp in slices keeps the temporaries small
    step = 1 << 27
    for a in range(0, total, step):
        b = min(total, a + step)
        z[a:b] = torch.ldexp(z[a:b], e[a:b].to(dtype))
    return z


def normal_like_torch(shape, dtype, seed: int = 4, device="cuda"):
    torch = _torch()
    g = _tgen(seed, device)
    return torch.randn(shape, generator=g, device=device, dtype=dtype)
