"""GPU parity of ragged batches (one persistent launch after the classifier):
every mapping (thread/warp/block thresholds, block size, grid) gives the
oracle's bits; graph replay; zero-length vectors; bad offsets are skipped and
reported without a fault; the autotuner picks a valid mapping."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_bits, cuda_device, f64_range_edges, f64_small_range_edges
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


def _batch(f, count, seed, nmax=4096, kind="mixture"):
    dt = DT[f]
    lengths = synth.ragged_lengths(count, seed=seed, kind=kind, nmax=nmax)
    # zero-length vectors, length 1, and a few long ones beyond the register paths
    lengths[::997] = 0
    lengths[5::1013] = 1
    lengths[7] = 6000
    lengths[11] = 20000
    off = synth.offsets_from_lengths(lengths)
    x = synth.ragged_values(lengths, dt, seed=seed)
    # a zero vector of each small length, NaNs, subnormals
    for i, n in ((12, 2), (13, 3), (14, 4), (15, 9), (16, 100)):
        lengths_i = off[i + 1] - off[i]
        if lengths_i >= n:
            x[off[i]:off[i + 1]] = 0
    x[off[20]] = np.nan
    x[off[21]:off[22]] = np.finfo(dt).smallest_subnormal
    return lengths, off, x


MAPPINGS = [(8, 8192, 256, 0), (4, 16, 256, 0), (4, 256, 128, 0), (16, 512, 256, 7), (5, 32, 128, 1),
            (16, 1024, 128, 0), (4, 4, 256, 3)]


@pytest.mark.parametrize("f", ["f32", "f64"])
def test_ragged_all_mappings(dev, f):
    from paper_1606_06508_gb300 import api
    lengths, off, x = _batch(f, 20011, seed=3)
    oy, orr, oh, oc = oracle.normalize(x, dim=0, offsets=off)
    xt, offt = _to(dev, x), _to(dev, off)
    plan = api.Plan(len(lengths), xt.dtype)
    for m in MAPPINGS:
        plan.set_mapping(*m)
        for graphs in (True, False):
            plan.set_graphs(graphs)
            y, r, h, c = api.normalize(xt, offt, return_norm=True, save=True, plan=plan)
            tag = f"{f} mapping={m} graphs={graphs}"
            assert_bits(_np(y), oy, tag + " y")
            assert_bits(_np(r), orr, tag + " norm")
            assert_bits(_np(h), oh, tag + " h")
            assert_bits(_np(c), oc, tag + " code")
    assert plan.query_status() == 0


@pytest.mark.parametrize("f", ["f32", "f64"])
def test_ragged_backward_all_mappings(dev, f):
    from paper_1606_06508_gb300 import api
    dt = DT[f]
    lengths, off, x = _batch(f, 7001, seed=4, nmax=3000)
    g = synth.normal_like(x.shape, dt, seed=44)
    oy, orr, oh, oc = oracle.normalize(x, dim=0, offsets=off)
    og = oracle.backward(oy, g, oh, oc, dim=0, offsets=off)
    xt, offt, gt = _to(dev, x), _to(dev, off), _to(dev, g)
    plan = api.Plan(len(lengths), xt.dtype)
    for m in MAPPINGS[:4]:
        plan.set_mapping(*m)
        y, h, c = api.normalize(xt, offt, save=True, plan=plan)
        gr = api.normalize_backward(y, gt, h, c, offt, plan=plan)
        assert_bits(_np(gr), og, f"{f} backward mapping={m}")


def test_ragged_f64_backward_over_the_exponent_range(dev):
    """binary64 ragged backward with inputs and upstream gradients over the
    whole exponent range, on thread, group and warp items: the products on
    the integer pipes are taken vector by vector (the range tests of the
    warp, group and thread backward), so vectors on both sides of every test
    meet in one batch; every gradient against the oracle, under the default
    mapping and one with thread_max 4."""
    from paper_1606_06508_gb300 import api
    rng = np.random.default_rng(23)
    count = 6007
    lengths = synth.ragged_lengths(count, seed=23, kind="loguniform", nmax=1024)
    off = synth.offsets_from_lengths(lengths)
    sx = rng.integers(-1000, 1001, size=count)
    x = rng.standard_normal(int(off[-1])) * np.ldexp(1.0, np.repeat(sx, lengths))
    sg = rng.choice(np.array([-1074, -1060, -1022, -1000, -900, -600, -300, 0, 300, 600, 900, 1000, 1015]), count)
    g = rng.standard_normal(int(off[-1])) * np.ldexp(1.0, np.repeat(sg, lengths))
    heads = off[:-1][lengths > 0]
    g[heads[::7]] = 2.0 ** 1000
    g[heads[1::7]] = 5e-324
    x[off[5]:off[6]] = 0
    oy, orr, oh, oc = oracle.normalize(x, dim=0, offsets=off)
    og = oracle.backward(oy, g, oh, oc, dim=0, offsets=off)
    xt, offt, gt = _to(dev, x), _to(dev, off), _to(dev, g)
    plan = api.Plan(count, xt.dtype)
    for m in (None, (4, 8192, 256, 0)):
        if m:
            plan.set_mapping(*m)
        y, h, c = api.normalize(xt, offt, save=True, plan=plan)
        assert_bits(_np(y), oy, f"f64 exponent range forward mapping={m}")
        gr = api.normalize_backward(y, gt, h, c, offt, plan=plan)
        assert_bits(_np(gr), og, f"f64 exponent range backward mapping={m}")
    assert plan.query_status() == 0


def test_graph_replay_with_new_buffers(dev):
    """Calls with other x / y buffers on the same plan re-record the graph."""
    from paper_1606_06508_gb300 import api
    plan = None
    for seed in (1, 2, 3):
        lengths, off, x = _batch("f32", 5003, seed=seed, nmax=1500)
        if plan is None:
            plan = api.Plan(len(lengths))
        y = api.normalize(_to(dev, x), _to(dev, off), plan=plan)
        assert_bits(_np(y), oracle.normalize(x, dim=0, offsets=off)[0], f"replay seed={seed}")


def test_norm_only_ragged(dev):
    from paper_1606_06508_gb300 import api
    lengths, off, x = _batch("f64", 3001, seed=9, nmax=5000)
    r = api.normalize(_to(dev, x), _to(dev, off), norm_only=True)
    assert_bits(_np(r), oracle.normalize(x, dim=0, offsets=off)[1], "ragged norm only")


def test_bad_offsets_reported_not_faulting(dev):
    """Decreasing offsets, a length beyond 2^20 and an end beyond the capacity
    are skipped and reported; the other vectors are still normalized."""
    import torch
    from paper_1606_06508_gb300 import _lib as L
    from paper_1606_06508_gb300 import api
    lengths = np.array([3, 5, 4, 7, 2, 9], dtype=np.int64)
    off = synth.offsets_from_lengths(lengths)
    x = synth.ragged_values(lengths, np.float32, seed=1)
    total = int(off[-1])
    bad = off.copy()
    bad[2] = bad[3] + 1          # vector 2 gets a negative length (vector 1 then overlaps vector 3)
    xt = _to(dev, x)
    plan = api.Plan(len(lengths), torch.float32, capacity=total)
    y = torch.zeros_like(xt)
    api.normalize(xt, _to(dev, bad), out=y, plan=plan)
    assert plan.query_status() == L.NGB_ERR_BAD_OFFSETS
    assert plan.query_status() == L.NGB_OK  # cleared by the query
    oy = oracle.normalize(x, dim=0, offsets=off)[0]
    good = [0, 4, 5]  # vectors that no other vector overlaps
    for i in good:
        assert_bits(_np(y)[off[i]:off[i + 1]], oy[off[i]:off[i + 1]], f"vector {i}")
    # an end beyond the capacity
    bad2 = off.copy()
    bad2[-1] = total + 10
    api.normalize(xt, _to(dev, bad2), out=y, plan=plan)
    assert plan.query_status() == L.NGB_ERR_BAD_OFFSETS
    # offsets[0] != 0 with validation
    bad3 = off + 0
    bad3[0] = 1
    api.normalize(xt, _to(dev, bad3), out=y, plan=plan, validate_offsets=True)
    assert plan.query_status() == L.NGB_ERR_BAD_OFFSETS
    api.normalize(xt, _to(dev, off), out=y, plan=plan, validate_offsets=True)
    assert plan.query_status() == L.NGB_OK


def test_plan_mismatch_and_missing(dev):
    import torch
    from paper_1606_06508_gb300 import _lib as L
    lengths, off, x = _batch("f32", 100, seed=2, nmax=50)
    xt, offt = _to(dev, x), _to(dev, off)
    st = L.normalize_f32(xt.data_ptr(), xt.data_ptr(), None, None, None, 100, 0, offt.data_ptr(), None, 0, 0)
    assert st == L.NGB_ERR_NO_PLAN
    st, p = L.ngb_plan_create(99, 4, 0)
    assert st == 0
    st = L.normalize_f32(xt.data_ptr(), xt.data_ptr(), None, None, None, 100, 0, offt.data_ptr(), p, 0, 0)
    assert st == L.NGB_ERR_NO_PLAN
    L.ngb_plan_destroy(p)
    torch.cuda.synchronize()


@pytest.mark.parametrize("f", ["f32", "f64"])
def test_autotune(dev, f, tmp_path):
    from paper_1606_06508_gb300 import api
    lengths, off, x = _batch(f, 30011, seed=6)
    xt, offt = _to(dev, x), _to(dev, off)
    plan = api.Plan(len(lengths), xt.dtype)
    cache = str(tmp_path / "tune.txt")
    m = plan.autotune(offt, cache)
    assert 4 <= m[0] <= 16 and m[0] <= m[1] <= (1 << 20) and m[2] in (128, 256)
    plan2 = api.Plan(len(lengths), xt.dtype)
    assert plan2.autotune(offt, cache) == m  # read back from the cache
    y = api.normalize(xt, offt, plan=plan)
    assert_bits(_np(y), oracle.normalize(x, dim=0, offsets=off)[0], f"{f} autotuned")


def test_ragged_f64_integer_pipe_limits(dev):
    """Warp and block items of a ragged binary64 batch whose components sit at
    the limits of the integer-pipe scale and square (see
    gpu_util.f64_range_edges), under two mappings."""
    from paper_1606_06508_gb300 import api
    rng = np.random.default_rng(12)
    lengths = rng.integers(17, 3000, size=600).astype(np.int64)
    lengths[::50] = 9000
    off = synth.offsets_from_lengths(lengths)
    x = np.empty(int(off[-1]))
    for i, n in enumerate(lengths):
        x[off[i]:off[i + 1]] = f64_range_edges(3, int(n), seed=i)[i % 3]
    oy, orr, oh, oc = oracle.normalize(x, dim=0, offsets=off)
    xt, offt = _to(dev, x), _to(dev, off)
    plan = api.Plan(len(lengths), xt.dtype)
    for m in ((8, 8192, 256, 0), (8, 1024, 128, 0)):
        plan.set_mapping(*m)
        y, r, h, c = api.normalize(xt, offt, return_norm=True, save=True, plan=plan)
        tag = f"f64 limits mapping={m}"
        assert_bits(_np(y), oy, tag + " y")
        assert_bits(_np(r), orr, tag + " norm")
        assert_bits(_np(c), oc, tag + " code")


def test_ragged_small_f64_integer_pipe_limits(dev):
    """Thread items of lengths 1-4 (one integer-pipe form for every length, the
    hardware steps per length outside its range) at the limits of
    gpu_util.f64_small_range_edges, under two mappings, with the backward."""
    from paper_1606_06508_gb300 import api
    rng = np.random.default_rng(13)
    lengths = rng.integers(1, 5, size=12000).astype(np.int64)
    off = synth.offsets_from_lengths(lengths)
    pools = {n: f64_small_range_edges(int(np.count_nonzero(lengths == n)), n, seed=30 + n) for n in range(1, 5)}
    used = {n: 0 for n in range(1, 5)}
    x = np.empty(int(off[-1]))
    for i, n in enumerate(lengths):
        x[off[i]:off[i + 1]] = pools[int(n)][used[int(n)]]
        used[int(n)] += 1
    g = rng.standard_normal(x.size)
    oy, orr, oh, oc = oracle.normalize(x, dim=0, offsets=off)
    og = oracle.backward(oy, g, oh, oc, dim=0, offsets=off)
    xt, offt, gt = _to(dev, x), _to(dev, off), _to(dev, g)
    plan = api.Plan(len(lengths), xt.dtype)
    for m in ((16, 8192, 256, 0), (4, 1024, 128, 3)):
        plan.set_mapping(*m)
        y, r, h, c = api.normalize(xt, offt, return_norm=True, save=True, plan=plan)
        tag = f"f64 small limits mapping={m}"
        assert_bits(_np(y), oy, tag + " y")
        assert_bits(_np(r), orr, tag + " norm")
        assert_bits(_np(h), oh, tag + " saved_h")
        assert_bits(_np(c), oc, tag + " code")
        gr = api.normalize_backward(y, gt, h, c, offt, plan=plan)
        assert_bits(_np(gr), og, tag + " grad")


@pytest.mark.parametrize("f", ["f32", "f64"])
def test_ragged_without_elements(dev, f):
    """A ragged batch whose element arrays are NULL (every vector empty, as a
    zero-element torch tensor gives): accepted, norms +0 and code 'zero' for
    the empty vectors; a vector of positive length in such a batch is skipped
    and reported as bad offsets, its outputs untouched; the backward call
    with NULL y, g and grad writes nothing and reports the same."""
    import torch
    from paper_1606_06508_gb300 import _lib as L
    from paper_1606_06508_gb300 import api
    td = torch.float32 if f == "f32" else torch.float64
    fwd = L.normalize_f32 if f == "f32" else L.normalize_f64
    bwd = L.normalize_backward_f32 if f == "f32" else L.normalize_backward_f64
    stream = torch.cuda.current_stream().cuda_stream
    for lengths, bad in (([0], False), ([0, 0, 0], False), ([0, 3, 0], True)):
        count = len(lengths)
        off = _to(dev, synth.offsets_from_lengths(np.array(lengths, np.int64)))
        plan = api.Plan(count, td)
        r = torch.full((count,), float("nan"), dtype=td, device=dev)
        h = torch.full((count,), float("nan"), dtype=td, device=dev)
        c = torch.full((count,), 77, dtype=torch.int8, device=dev)
        for graphs in (True, False):
            plan.set_graphs(graphs)
            st = fwd(None, None, r.data_ptr(), h.data_ptr(), c.data_ptr(), count, 0, off.data_ptr(), plan.handle, 0,
                     stream)
            assert st == L.NGB_OK, L.last_error()
            assert plan.query_status() == (L.NGB_ERR_BAD_OFFSETS if bad else L.NGB_OK)
            empty = np.array(lengths) == 0
            rn, hn, cn = _np(r), _np(h), _np(c)
            assert np.all(rn[empty] == 0) and not np.any(np.signbit(rn[empty])) and np.all(hn[empty] == 0)
            assert np.all(cn[empty] == L.NGB_CODE_ZERO)
            assert np.all(np.isnan(rn[~empty])) and np.all(cn[~empty] == 77)
            st = bwd(None, None, h.data_ptr(), c.data_ptr(), None, count, 0, off.data_ptr(), plan.handle, 0, stream)
            assert st == L.NGB_OK, L.last_error()
            assert plan.query_status() == (L.NGB_ERR_BAD_OFFSETS if bad else L.NGB_OK)
        # the torch-facing helper on an empty values tensor
        y = api.normalize(torch.empty(0, dtype=td, device=dev), off, plan=plan)
        assert y.numel() == 0
        plan.close()
