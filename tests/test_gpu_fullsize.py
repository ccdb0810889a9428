"""Full-size workloads, in the launch configuration the benchmark times: inputs
are generated on the device, the whole batch is normalized, and EVERY output
(y, norm, saved h, code; the gradient for the forward + backward workload) is
compared bit for bit with the oracle on the same inputs, the oracle running
on all host cores over contiguous vector ranges."""
import os

import numpy as np
import pytest

import oracle
from gpu_util import assert_bits, cuda_device
from paper_1606_06508_gb300 import synth

pytestmark = pytest.mark.gpu

THREADS = max(1, len(os.sched_getaffinity(0)))


@pytest.fixture(scope="module")
def dev():
    d = cuda_device()
    import __graft_entry__
    __graft_entry__.build()
    return d


def _np(t):
    return t.detach().cpu().numpy()


def _compare_all(what, gpu, ref):
    for name, a, b in zip(("y", "norm", "saved_h", "saved_code"), gpu, ref):
        if a is not None:
            assert_bits(_np(a).reshape(-1), b.reshape(-1), f"{what} {name} (every vector)")


def test_config0_vectors3_f64_full(dev):
    """65,536 binary64 3-vectors (e in [-30, 30]) and the 64 edge vectors."""
    import torch
    from paper_1606_06508_gb300 import api
    xh = synth.vectors3_f64(65536, seed=0)
    assert xh.shape == (65600, 3)
    y, r, h, c = api.normalize(torch.from_numpy(xh).to(dev), return_norm=True, save=True)
    torch.cuda.synchronize()
    _compare_all("65,600 x 3 f64", (y, r, h, c), oracle.normalize_threads(xh.reshape(-1), 3, threads=THREADS))


def test_config1_quaternions_full(dev):
    import torch
    from paper_1606_06508_gb300 import api
    count = 1 << 26
    x = synth.quaternions_f32_torch(count, seed=1, device=dev)
    y, r, h, c = api.normalize(x, return_norm=True, save=True)
    torch.cuda.synchronize()
    ref = oracle.normalize_threads(_np(x).reshape(-1), 4, threads=THREADS)
    _compare_all("2^26 quaternions", (y, r, h, c), ref)


@pytest.mark.parametrize("f,count", [("f32", 1 << 20), ("f64", 1 << 19)])
def test_config2_rows_full(dev, f, count):
    import torch
    from paper_1606_06508_gb300 import api
    dt = torch.float32 if f == "f32" else torch.float64
    x = synth.rows_torch(count, 256, dt, seed=2, device=dev)
    y, r, h, c = api.normalize(x, return_norm=True, save=True)
    torch.cuda.synchronize()
    ref = oracle.normalize_threads(_np(x).reshape(-1), 256, threads=THREADS)
    _compare_all(f"{f} rows of 256", (y, r, h, c), ref)


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
    xh, offh = _np(x), _np(off)
    del x
    ref = oracle.normalize_threads(xh, 0, offh, threads=THREADS)
    del xh
    _compare_all(f"{f} ragged 4M", (y, r, h, c), ref)


def test_config4_forward_backward_full(dev):
    import torch
    from paper_1606_06508_gb300 import api
    # 2^24 binary32 quaternions
    count = 1 << 24
    x = synth.quaternions_f32_torch(count, seed=4, device=dev)
    g = synth.normal_like_torch((count, 4), torch.float32, seed=40, device=dev)
    y, h, c = api.normalize(x, save=True)
    grad = api.normalize_backward(y, g, h, c)
    torch.cuda.synchronize()
    oy, orr, oh, oc = oracle.normalize_threads(_np(x).reshape(-1), 4, threads=THREADS)
    _compare_all("2^24 quaternions fwd", (y, None, h, c), (oy, orr, oh, oc))
    og = oracle.backward_threads(oy, _np(g).reshape(-1), oh, oc, dim=4, threads=THREADS)
    assert_bits(_np(grad).reshape(-1), og, "2^24 quaternions grad (every vector)")
    # 500,000 binary64 ragged vectors, lengths log-uniform in [2, 1024]
    count = 500_000
    lengths = synth.ragged_lengths_torch(count, seed=4, kind="loguniform", nmax=1024, device=dev)
    off = synth.offsets_from_lengths_torch(lengths)
    v = synth.ragged_values_torch(lengths, torch.float64, seed=4)
    gv = synth.normal_like_torch(v.shape, torch.float64, seed=41, device=dev)
    plan = api.Plan(count, torch.float64)
    y, r, h, c = api.normalize(v, off, return_norm=True, save=True, plan=plan)
    grad = api.normalize_backward(y, gv, h, c, off, plan=plan)
    torch.cuda.synchronize()
    assert plan.query_status() == 0
    offh = _np(off)
    oy, orr, oh, oc = oracle.normalize_threads(_np(v), 0, offh, threads=THREADS)
    _compare_all("f64 ragged 500k fwd", (y, r, h, c), (oy, orr, oh, oc))
    og = oracle.backward_threads(oy, _np(gv), oh, oc, dim=0, offsets=offh, threads=THREADS)
    assert_bits(_np(grad), og, "f64 ragged 500k grad (every vector)")
