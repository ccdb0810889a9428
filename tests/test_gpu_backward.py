"""GPU parity of the backward pass (dense and ragged) with the oracle, the
autograd Function, and the adjoint against FP64 central differences."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_bits, cuda_device
from paper_1606_06508_gb300 import synth

pytestmark = pytest.mark.gpu

DT = {"f32": np.float32, "f64": np.float64}


@pytest.fixture(scope="module")
def dev():
    d = cuda_device()
    import __graft_entry__
    __graft_entry__.build()
    return d


def _to(dev, a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def _np(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("f", ["f32", "f64"])
@pytest.mark.parametrize("dim", [1, 2, 3, 4, 5, 9, 16, 17, 33, 64, 65, 100, 128, 129, 256, 257, 1000, 1023, 1500, 2500,
                                 4096, 5000])
def test_dense_backward(dev, f, dim):
    from paper_1606_06508_gb300 import api
    dt = DT[f]
    count = max(3, min(70001, 300000 // dim))
    x = synth.rows(count, dim, dt, seed=30 + dim, smax=100 if f == "f32" else 900)
    x[0] = 0
    g = synth.normal_like(x.shape, dt, seed=31)
    xt, gt = _to(dev, x), _to(dev, g)
    y, h, c = api.normalize(xt, save=True)
    grad = api.normalize_backward(y, gt, h, c)
    oy, _, oh, oc = oracle.normalize(x.reshape(-1), dim=dim)
    og = oracle.backward(oy, g.reshape(-1), oh, oc, dim=dim)
    assert_bits(_np(grad), og, f"{f} d={dim} backward")
    # in place: grad written over g
    api.normalize_backward(y, gt, h, c, out=gt)
    assert_bits(_np(gt), og, f"{f} d={dim} backward in place")


def test_autograd_function(dev):
    import torch
    from paper_1606_06508_gb300 import api
    x = synth.quaternions_f32(10007, seed=1)
    g = synth.normal_like(x.shape, np.float32, seed=2)
    xt = _to(dev, x).requires_grad_(True)
    y = api.NormalizeFn.apply(xt)
    (y * _to(dev, g)).sum().backward()
    oy, _, oh, oc = oracle.normalize(x.reshape(-1), dim=4)
    assert_bits(_np(y), oy, "autograd forward")
    assert_bits(_np(xt.grad), oracle.backward(oy, g.reshape(-1), oh, oc, dim=4), "autograd backward")
    # ragged
    lengths = synth.ragged_lengths(3001, seed=5, kind="loguniform", nmax=1024)
    off = synth.offsets_from_lengths(lengths)
    v = synth.ragged_values(lengths, np.float64, seed=5)
    gv = synth.normal_like(v.shape, np.float64, seed=6)
    vt = _to(dev, v).requires_grad_(True)
    yr = api.NormalizeFn.apply(vt, _to(dev, off))
    (yr * _to(dev, gv)).sum().backward()
    oy, _, oh, oc = oracle.normalize(v, dim=0, offsets=off)
    assert_bits(_np(vt.grad), oracle.backward(oy, gv, oh, oc, dim=0, offsets=off), "autograd ragged backward")
    torch.cuda.synchronize()


def test_adjoint_central_differences(dev):
    """The GPU adjoint against FP64 central differences (step 1e-6 |v|) of the
    oracle's binary64 forward, on sampled vectors of both families."""
    from paper_1606_06508_gb300 import api
    rng = np.random.default_rng(7)
    # binary32 quaternions, upcast for the differences
    q = synth.quaternions_f32(20000, seed=1)
    q = q[np.all(np.abs(q) < 1e30, axis=1) & np.all(np.abs(q) > 1e-30, axis=1)]
    g = synth.normal_like(q.shape, np.float32, seed=3)
    y, h, c = api.normalize(_to(dev, q), save=True)
    grad = _np(api.normalize_backward(y, _to(dev, g), h, c))
    for i in rng.choice(q.shape[0], 512, replace=False):
        xi = q[i].astype(np.float64)
        r = float(np.linalg.norm(xi))
        step = 1e-6 * r
        fd = np.empty(4)
        for k in range(4):
            xp, xm = xi.copy(), xi.copy()
            xp[k] += step
            xm[k] -= step
            fd[k] = np.dot(g[i].astype(np.float64), oracle.normalize(xp, dim=4)[0] - oracle.normalize(xm, dim=4)[0]) \
                / (2 * step)
        scale = np.linalg.norm(g[i].astype(np.float64)) / r
        assert np.max(np.abs(fd - grad[i])) <= 2e-6 * scale, (i, fd, grad[i])
    # binary64 ragged
    lengths = synth.ragged_lengths(2000, seed=8, kind="loguniform", nmax=200)
    off = synth.offsets_from_lengths(lengths)
    v = synth.ragged_values(lengths, np.float64, seed=8)
    gv = synth.normal_like(v.shape, np.float64, seed=9)
    y, h, c = api.normalize(_to(dev, v), _to(dev, off), save=True)
    grad = _np(api.normalize_backward(y, _to(dev, gv), h, c, _to(dev, off)))
    for i in rng.choice(len(lengths), 64, replace=False):
        a, b = off[i], off[i + 1]
        xi = v[a:b]
        n = b - a
        r = float(np.linalg.norm(xi))
        step = 1e-6 * r
        fd = np.empty(n)
        for k in range(n):
            xp, xm = xi.copy(), xi.copy()
            xp[k] += step
            xm[k] -= step
            fd[k] = np.dot(gv[a:b], oracle.normalize(xp, dim=n)[0] - oracle.normalize(xm, dim=n)[0]) / (2 * step)
        scale = np.linalg.norm(gv[a:b]) / r
        assert np.max(np.abs(fd - grad[a:b])) <= 1e-7 * scale, i


@pytest.mark.parametrize("dim", [20, 300, 1500, 5000])
def test_f64_backward_integer_pipe_limits(dev, dim):
    """binary64 backward where the products y_k g_k and y_k dot leave or stay
    in the range of the integer-pipe product: tiny and huge g components, tiny
    y components (from inputs at the forward's limits), zero g, g with one
    huge entry; dense rows and a ragged batch of the same vectors."""
    from gpu_util import f64_range_edges
    from paper_1606_06508_gb300 import api
    rng = np.random.default_rng(dim)
    count = max(40, min(600, 200000 // dim))
    x = f64_range_edges(count, dim, seed=dim)
    g = rng.standard_normal((count, dim))
    for i in range(count):
        kind = i % 6
        if kind == 1:
            g[i] *= 2.0 ** 600              # products near the top of the range with huge dot
        elif kind == 2:
            g[i] *= 2.0 ** -600             # tiny products
        elif kind == 3:
            g[i, int(rng.integers(dim))] = 2.0 ** -1060  # a subnormal g component
        elif kind == 4:
            g[i] = 0.0                      # dot = 0
        elif kind == 5:
            g[i, int(rng.integers(dim))] = 2.0 ** 1000
    xt, gt = _to(dev, x), _to(dev, g)
    y, h, c = api.normalize(xt, save=True)
    grad = api.normalize_backward(y, gt, h, c)
    oy, _, oh, oc = oracle.normalize(x.reshape(-1), dim=dim)
    og = oracle.backward(oy, g.reshape(-1), oh, oc, dim=dim)
    assert_bits(_np(grad), og, f"f64 d={dim} backward at the integer-pipe limits")
    # the same vectors as a ragged batch (warp list)
    off = np.arange(count + 1, dtype=np.int64) * dim
    offt = _to(dev, off)
    plan = api.Plan(count, xt.dtype)
    plan.set_mapping(8, 8192, 256, 0)
    yr, hr, cr = api.normalize(xt.reshape(-1), offt, save=True, plan=plan)
    gr = api.normalize_backward(yr, gt.reshape(-1), hr, cr, offt, plan=plan)
    assert_bits(_np(gr), og, f"f64 d={dim} ragged backward at the integer-pipe limits")
