"""Helpers for the parity tests (GPU and host builds): bitwise comparison with
NaN as a class, binary64 inputs at the limits of the integer-pipe steps, and
the two-component binary32 exponent grid."""
import numpy as np
import pytest


def bits_equal(gpu, ref):
    """(number of mismatches, first mismatching flat index or -1).  Equal means
    the same bit pattern, except that any NaN matches any NaN."""
    a = np.ascontiguousarray(np.asarray(gpu)).reshape(-1)
    b = np.ascontiguousarray(np.asarray(ref)).reshape(-1)
    assert a.shape == b.shape and a.dtype == b.dtype, (a.shape, b.shape, a.dtype, b.dtype)
    if a.dtype.kind == "f":
        ui = np.uint32 if a.dtype == np.float32 else np.uint64
        nan = np.isnan(a) & np.isnan(b)
        diff = (a.view(ui) != b.view(ui)) & ~nan
    else:
        diff = a != b
    bad = np.flatnonzero(diff)
    return bad.size, (int(bad[0]) if bad.size else -1)


def assert_bits(gpu, ref, what=""):
    n, i = bits_equal(gpu, ref)
    if n:
        a = np.asarray(gpu).reshape(-1)
        b = np.asarray(ref).reshape(-1)
        pytest.fail(f"{what}: {n} values differ from the oracle; first at {i}: gpu={a[i]!r} oracle={b[i]!r}")


def cuda_device():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch.device("cuda:0")


def f64_range_edges(count, dim, seed):
    """binary64 vectors whose smallest nonzero component sits on, just below or
    just above the lower limit of the integer-pipe scale and square (|c x| =
    2^-511 after the factor c = 1, sigma_min = 2^592 or sigma_max = 2^-523),
    next to vectors that stay inside it, with zeros, subnormals and the smallest
    normal number mixed in."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((count, dim))
    below = np.nextafter(2.0 ** -511, 0.0)
    for i in range(count):
        kind = i % 3
        if kind == 0:      # c = 1: max near 1, limit 2^-511
            edge = [2.0 ** -511, below, np.nextafter(2.0 ** -511, 1.0), 2.0 ** -600, 5e-324, 0.0]
        elif kind == 1:    # sigma_max: max near 2^600, limit 2^12
            x[i] *= 2.0 ** 600
            edge = [2.0 ** 12, np.nextafter(2.0 ** 12, 0.0), 3.0 * 2.0 ** 11, 1.0, 2.0 ** -1022, 0.0]
        else:              # sigma_min: max near 2^-500, subnormal components leave the integer path
            x[i] *= 2.0 ** -500
            edge = [2.0 ** -1022, np.nextafter(2.0 ** -1022, 0.0), 5e-324, 2.0 ** -700, 0.0, 2.0 ** -1000]
        j = (i // 3) % (len(edge) + 1)
        if j < len(edge):  # the last choice leaves the vector untouched
            x[i, int(rng.integers(dim))] = edge[j]
            if j % 2:
                x[i, int(rng.integers(dim))] = -edge[j]
    return x


def f64_small_range_edges(count, dim, seed):
    """binary64 vectors of dim <= 4 at the limits of the integer-pipe form of
    Normalize2D/3D/4D, whose factor comes from the n <= 4 row of Table 2
    (tau_min = 2^-482, tau_max = 2^510, sigma_min = 2^592, sigma_max = 2^-514):
    the smallest nonzero component on, just below or just above |c x| =
    2^-511; the largest magnitude on and next to tau_min and tau_max; norms
    r^ = r~ / c at and beyond the overflow threshold; zeros of both signs,
    subnormals and the smallest normal number."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((count, dim))
    up = lambda v: np.nextafter(v, np.inf)  # noqa: E731
    dn = lambda v: np.nextafter(v, 0.0)  # noqa: E731
    for i in range(count):
        kind = i % 5
        edge = []
        if kind == 0:      # c = 1: max near 1, limit 2^-511
            edge = [2.0 ** -511, dn(2.0 ** -511), up(2.0 ** -511), 2.0 ** -600, 5e-324, 0.0, -0.0]
        elif kind == 1:    # sigma_max: max near 2^600, limit 2^3
            x[i] *= 2.0 ** 600
            edge = [8.0, dn(8.0), 12.0, 1.0, 2.0 ** -1022, 0.0, -0.0]
        elif kind == 2:    # sigma_min: max near 2^-500; subnormal components leave the integer form
            x[i] *= 2.0 ** -500
            edge = [2.0 ** -1022, dn(2.0 ** -1022), 5e-324, 2.0 ** -700, 0.0, 2.0 ** -1000, -0.0]
        elif kind == 3:    # the largest magnitude on and next to tau_min and tau_max
            t = [2.0 ** -482, dn(2.0 ** -482), up(2.0 ** -482), 2.0 ** 510, up(2.0 ** 510),
                 dn(2.0 ** 510)][(i // 5) % 6]
            x[i] = t * rng.uniform(0.01, 1.0, size=dim) * np.where(rng.integers(0, 2, size=dim) == 1, -1.0, 1.0)
            x[i, int(rng.integers(dim))] = t
        else:              # sigma_max, norms near 2^1024: some overflow to infinity
            e = rng.integers(1020, 1024, size=dim).astype(np.int32)
            x[i] = np.ldexp(rng.uniform(1.0, 2.0, size=dim), e) * np.where(rng.integers(0, 2, size=dim) == 1, -1.0, 1.0)
        j = (i // 5) % (len(edge) + 1)
        if j < len(edge):  # the last choice leaves the vector untouched
            x[i, int(rng.integers(dim))] = edge[j]
            if j % 2:
                x[i, int(rng.integers(dim))] = -edge[j]
    return x


def full_grid_two_f32(signs=(1.0,)):
    """Every exponent pair (e1, e2) in [-149, 127]^2 of binary32, with the
    mantissas {1, 1.5, 2 - 2^-23} for each component and the sign patterns of
    x2 (x1's sign is covered by the sign-flip invariance)."""
    es = np.arange(-149, 128)
    mants = np.array([1.0, 1.5, 2.0 - 2.0 ** -23])
    e1, e2, m1, m2, sg = np.meshgrid(es, es, mants, mants, np.array(signs), indexing="ij")
    x1 = np.ldexp(m1, e1).reshape(-1)
    x2 = (sg * np.ldexp(m2, e2)).reshape(-1)
    return np.stack([x1, x2], axis=1).astype(np.float32)
