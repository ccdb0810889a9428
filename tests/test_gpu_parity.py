"""GPU parity: the CUDA library against the oracle, element by element, bit for
bit (NaN compared as a class), through the C ABI (via the torch helpers,
which only marshal arguments).  Sizes span several tiles with a ragged tail;
the full-size workloads are checked on sampled vectors in test_gpu_fullsize.py.
"""
import numpy as np
import pytest

import oracle
from gpu_util import assert_bits, cuda_device, f64_range_edges, f64_small_range_edges, full_grid_two_f32
from paper_1606_06508_gb300 import synth

pytestmark = pytest.mark.gpu

DT = {"f32": np.float32, "f64": np.float64}


@pytest.fixture(scope="module")
def dev():
    d = cuda_device()
    import __graft_entry__
    __graft_entry__.build()
    return d


def _api():
    from paper_1606_06508_gb300 import api
    return api


def _to(dev, a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def _np(t):
    return t.detach().cpu().numpy()


def _specials(x, dt, rng):
    """Plant zeros, NaNs, infinities, subnormals and extremes in some vectors."""
    fi = np.finfo(dt)
    n = x.shape[1]
    vals = [0.0, -0.0, np.nan, np.inf, -np.inf, float(fi.max), float(fi.tiny), float(fi.smallest_subnormal),
            -float(fi.smallest_subnormal) * 3, 1.0]
    cnt = x.shape[0]
    for j in range(min(cnt // 4, 4000)):
        i = int(rng.integers(cnt))
        k = int(rng.integers(n))
        x[i, k] = vals[j % len(vals)]
    x[0] = 0
    x[1] = -0.0
    if cnt > 5:
        x[5] = 0
        x[5, n - 1] = float(fi.smallest_subnormal)
    return x


def _check_forward(dev, x, dim, flags=0, what=""):
    api = _api()
    xt = _to(dev, x)
    y, r, h, c = api.normalize(xt, return_norm=True, save=True, vector_semantics=bool(flags & 1))
    oy, orr, oh, oc = oracle.normalize(x.reshape(-1), dim=dim, flags=flags)
    assert_bits(_np(y), oy, f"{what} y")
    assert_bits(_np(r), orr, f"{what} norm")
    assert_bits(_np(h), oh, f"{what} saved_h")
    assert_bits(_np(c), oc, f"{what} saved_code")
    return y, h, c


@pytest.mark.parametrize("f", ["f32", "f64"])
@pytest.mark.parametrize("dim", [1, 2, 3, 4])
def test_small_dims(dev, f, dim):
    dt = DT[f]
    rng = np.random.default_rng(dim)
    count = 3 * 65536 + 123
    x = synth.vectors_f32(count, dim, seed=10 + dim) if f == "f32" else synth.vectors_f64(count, dim, seed=10 + dim)
    x = _specials(x, dt, rng)
    _check_forward(dev, x, dim, what=f"{f} d={dim}")
    if dim == 4:
        _check_forward(dev, x, dim, flags=1, what=f"{f} d=4 vector semantics")


def test_full_exponent_grid_two_components_f32(dev):
    """n = 2, binary32: every exponent pair in [-149, 127]^2, the mantissas
    {1, 1.5, 2 - 2^-23} for each component and the four sign patterns."""
    x = full_grid_two_f32(signs=(1.0, -1.0))
    x = np.concatenate([x, -x])
    _check_forward(dev, x, 2, what="f32 n=2 full exponent grid")


def test_quaternions_config_recipe(dev):
    x = synth.quaternions_f32(200003, seed=1)
    _check_forward(dev, x, 4, what="quaternions")


def test_config0_vectors3_f64(dev):
    x = synth.vectors3_f64(65536, seed=0)
    _check_forward(dev, x, 3, what="65600 x 3 binary64")


@pytest.mark.parametrize("f", ["f32", "f64"])
@pytest.mark.parametrize("dim", [1, 2, 3, 4])
def test_misaligned_and_inplace(dev, f, dim):
    """A base that is not 16-byte aligned takes the scalar-load path; y may equal x."""
    import torch
    api = _api()
    dt = DT[f]
    count = 70001
    x = synth.vectors_f32(count, dim, seed=3) if f == "f32" else synth.vectors_f64(count, dim, seed=3)
    buf = torch.empty(count * dim + 1, dtype=torch.float32 if f == "f32" else torch.float64, device=dev)
    buf[1:] = _to(dev, x.reshape(-1))
    xv = buf[1:].view(count, dim)
    y = api.normalize(xv)
    oy = oracle.normalize(x.reshape(-1), dim=dim)[0]
    assert_bits(_np(y), oy, "misaligned")
    api.normalize(xv, out=xv)  # in place
    assert_bits(_np(xv), oy, "in place")


@pytest.mark.parametrize("f", ["f32", "f64"])
@pytest.mark.parametrize("dim", [5, 7, 16, 17, 31, 32, 33, 64, 65, 100, 127, 128, 129, 132, 200, 252, 255, 256, 257, 512, 1000, 1024, 1025, 2048,
                                 3000, 4096, 4097, 20000])
def test_rows(dev, f, dim):
    dt = DT[f]
    count = max(3, min(2000, 400000 // dim))
    x = synth.rows(count, dim, dt, seed=2)
    rng = np.random.default_rng(dim)
    x = _specials(x, dt, rng)
    _check_forward(dev, x, dim, what=f"{f} rows d={dim}")


@pytest.mark.parametrize("f", ["f32", "f64"])
def test_rows_wide_values(dev, f):
    dt = DT[f]
    for dim in (6, 40, 256, 1500):
        x = synth.vectors_f32(300, dim, seed=dim) if f == "f32" else synth.vectors_f64(300, dim, seed=dim)
        _check_forward(dev, x, dim, what=f"{f} wide rows d={dim}")


@pytest.mark.parametrize("f", ["f32", "f64"])
def test_norm_only(dev, f):
    api = _api()
    dt = DT[f]
    for dim in (3, 4, 256, 3000):
        x = synth.rows(999, dim, dt, seed=5)
        r = api.normalize(_to(dev, x), norm_only=True)
        assert_bits(_np(r), oracle.normalize(x.reshape(-1), dim=dim)[1], f"norm only d={dim}")


def test_zero_count_and_empty(dev):
    import torch
    api = _api()
    x = torch.empty((0, 4), device=dev)
    y = api.normalize(x)
    assert y.shape == (0, 4)


@pytest.mark.parametrize("f", ["f32", "f64"])
def test_rotation(dev, f):
    api = _api()
    dt = DT[f]
    q = synth.quaternions_f32(70001, seed=8).astype(dt) if f == "f32" else synth.vectors_f64(70001, 4, seed=8)
    q[0] = 0
    q[3, 1] = np.nan
    R, r = api.normalize_to_rotation(_to(dev, q), return_norm=True)
    oR, orr = oracle.rotation(q)
    assert_bits(_np(R), oR, "rotation R")
    assert_bits(_np(r), orr, "rotation norm")


@pytest.mark.parametrize("dim", [5, 9, 17, 40, 256, 1000, 1024, 1025, 3000, 20000])
def test_f64_integer_pipe_limits(dev, dim):
    count = max(36, min(1200, 300000 // dim))
    x = f64_range_edges(count, dim, seed=dim)
    _check_forward(dev, x, dim, what=f"f64 integer-pipe limits d={dim}")


@pytest.mark.parametrize("dim", [1, 2, 3, 4])
def test_small_f64_integer_pipe_limits(dev, dim):
    """n <= 4 binary64 vectors at the limits of the integer-pipe form (and just
    outside it), through the 16-byte and the scalar-load kernels."""
    import torch
    api = _api()
    x = f64_small_range_edges(6000 + dim, dim, seed=20 + dim)
    _check_forward(dev, x, dim, what=f"f64 small limits d={dim}")
    if dim == 4:
        _check_forward(dev, x, dim, flags=1, what="f64 small limits d=4 vector semantics")
    count = x.shape[0]
    buf = torch.empty(count * dim + 1, dtype=torch.float64, device=dev)
    buf[1:] = _to(dev, x.reshape(-1))
    y = api.normalize(buf[1:].view(count, dim))
    assert_bits(_np(y), oracle.normalize(x.reshape(-1), dim=dim)[0], f"f64 small limits d={dim} misaligned")


@pytest.mark.parametrize("f", ["f32", "f64"])
@pytest.mark.parametrize("count", [1, 2, 3, 1001])
def test_rows_odd_counts(dev, f, count):
    """Row kernels that put several rows on one warp (half-warps, groups of 8
    or 16 lanes): counts that are not a multiple leave the last warp's later
    groups without a row of their own."""
    dt = DT[f]
    for dim in (20, 64, 100, 132, 256):
        x = synth.rows(count, dim, dt, seed=count + dim)
        _check_forward(dev, x, dim, what=f"{f} rows d={dim} count={count}")
