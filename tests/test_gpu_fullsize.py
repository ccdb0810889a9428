"""Full-size workloads, in the launch configuration the benchmark times: inputs
are generated on the device, the whole batch is normalized, and sampled
vectors (plus the first and last ones) are compared bit for bit with the
oracle on the same inputs; properties that hold at any size are checked on
every vector (finite outputs, unit length within the paper's bound, codes)."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_bits, cuda_device
from paper_1606_06508_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    d = cuda_device()
    import __graft_entry__
    __graft_entry__.build()
    return d


def _np(t):
    return t.detach().cpu().numpy()


def _sample(count, k, seed):
    rng = np.random.default_rng(seed)
    idx = np.unique(np.concatenate([np.arange(min(count, 300)), np.arange(max(0, count - 300), count),
                                    rng.choice(count, size=min(count, k), replace=False)]))
    return idx


def _unit_length_ok(y2d, u, bound_u):
    """| |y| - 1 | <= bound * u for every row (|y - x/r| <= bound u implies it)."""
    import torch
    n = torch.linalg.vector_norm(y2d.double(), dim=-1)
    return float(torch.max(torch.abs(n - 1)).item()) <= bound_u * u


def test_config1_quaternions_full(dev):
    import torch
    from paper_1606_06508_gb300 import api
    count = 1 << 26
    x = synth.quaternions_f32_torch(count, seed=1, device=dev)
    y, r, h, c = api.normalize(x, return_norm=True, save=True)
    torch.cuda.synchronize()
    assert bool(torch.isfinite(y).all()) and bool((r > 0).all()) and int(c.max()) <= 2
    assert _unit_length_ok(y, 2.0 ** -24, 5.001 + 1)
    idx = _sample(count, 1 << 16, 11)
    it = torch.from_numpy(idx).to(dev)
    xs = _np(x[it])
    oy, orr, oh, oc = oracle.normalize(xs.reshape(-1), dim=4)
    assert_bits(_np(y[it]).reshape(-1), oy, "2^26 quaternions y (sampled)")
    assert_bits(_np(r[it]), orr, "norm")
    assert_bits(_np(h[it]), oh, "h")
    assert_bits(_np(c[it]), oc, "code")


@pytest.mark.parametrize("f,count", [("f32", 1 << 20), ("f64", 1 << 19)])
def test_config2_rows_full(dev, f, count):
    import torch
    from paper_1606_06508_gb300 import api
    dt = torch.float32 if f == "f32" else torch.float64
    x = synth.rows_torch(count, 256, dt, seed=2, device=dev)
    y, r = api.normalize(x, return_norm=True)
    torch.cuda.synchronize()
    assert bool(torch.isfinite(y).all())
    u = 2.0 ** -24 if f == "f32" else 2.0 ** -53
    assert _unit_length_ok(y, u, 3.001 + 11)
    idx = _sample(count, 4096, 12)
    it = torch.from_numpy(idx).to(dev)
    xs = _np(x[it])
    oy, orr, _, _ = oracle.normalize(xs.reshape(-1), dim=256)
    assert_bits(_np(y[it]).reshape(-1), oy, f"{f} rows y (sampled)")
    assert_bits(_np(r[it]), orr, f"{f} rows norm (sampled)")


def _ragged_sample_check(dev, x, off_t, y, r, count, k, seed, what, h=None, c=None):
    import torch
    idx = _sample(count, k, seed)
    off = _np(off_t)
    # gather the sampled vectors into a packed batch
    starts, ends = off[idx], off[idx + 1]
    lens = ends - starts
    sub_off = synth.offsets_from_lengths(lens)
    gather = np.concatenate([np.arange(a, b) for a, b in zip(starts, ends)]).astype(np.int64)
    gt = torch.from_numpy(gather).to(dev)
    xs = _np(x[gt])
    oy, orr, oh, oc = oracle.normalize(xs, dim=0, offsets=sub_off)
    assert_bits(_np(y[gt]), oy, f"{what} y (sampled)")
    it = torch.from_numpy(idx).to(dev)
    assert_bits(_np(r[it]), orr, f"{what} norm (sampled)")
    if h is not None:
        assert_bits(_np(h[it]), oh, f"{what} h (sampled)")
        assert_bits(_np(c[it]), oc, f"{what} code (sampled)")
    return idx, gather, sub_off


@pytest.mark.parametrize("f", ["f32", "f64"])
def test_config3_ragged_full(dev, f):
    import torch
    from paper_1606_06508_gb300 import api
    dt = torch.float32 if f == "f32" else torch.float64
    count = 4_000_000
    lengths = synth.ragged_lengths_torch(count, seed=3, device=dev)
    off = synth.offsets_from_lengths_torch(lengths)
    x = synth.ragged_values_torch(lengths, dt, seed=3)
    plan = api.Plan(count, dt)
    plan.autotune(off)
    y, r, h, c = api.normalize(x, off, return_norm=True, save=True, plan=plan)
    torch.cuda.synchronize()
    assert plan.query_status() == 0
    assert bool(torch.isfinite(y).all()) and bool((r > 0).all())
    _ragged_sample_check(dev, x, off, y, r, count, 3000, 13, f"{f} ragged 4M", h, c)
    del x, y


def test_config4_forward_backward_full(dev):
    import torch
    from paper_1606_06508_gb300 import api
    # 2^24 binary32 quaternions
    count = 1 << 24
    x = synth.quaternions_f32_torch(count, seed=4, device=dev)
    g = synth.normal_like_torch((count, 4), torch.float32, seed=40, device=dev)
    y, h, c = api.normalize(x, save=True)
    grad = api.normalize_backward(y, g, h, c)
    idx = _sample(count, 1 << 15, 14)
    it = torch.from_numpy(idx).to(dev)
    oy, _, oh, oc = oracle.normalize(_np(x[it]).reshape(-1), dim=4)
    og = oracle.backward(oy, _np(g[it]).reshape(-1), oh, oc, dim=4)
    assert_bits(_np(grad[it]).reshape(-1), og, "2^24 quaternions grad (sampled)")
    # 500,000 binary64 ragged vectors, lengths log-uniform in [2, 1024]
    count = 500_000
    lengths = synth.ragged_lengths_torch(count, seed=4, kind="loguniform", nmax=1024, device=dev)
    off = synth.offsets_from_lengths_torch(lengths)
    v = synth.ragged_values_torch(lengths, torch.float64, seed=4)
    gv = synth.normal_like_torch(v.shape, torch.float64, seed=41, device=dev)
    plan = api.Plan(count, torch.float64)
    y, r, h, c = api.normalize(v, off, return_norm=True, save=True, plan=plan)
    grad = api.normalize_backward(y, gv, h, c, off, plan=plan)
    idx, gather, sub_off = _ragged_sample_check(dev, v, off, y, r, count, 3000, 15, "f64 ragged 500k", h, c)
    gt = torch.from_numpy(gather).to(dev)
    oy, _, oh, oc = oracle.normalize(_np(v[gt]), dim=0, offsets=sub_off)
    og = oracle.backward(oy, _np(gv[gt]), oh, oc, dim=0, offsets=sub_off)
    assert_bits(_np(grad[gt]), og, "f64 ragged 500k grad (sampled)")
