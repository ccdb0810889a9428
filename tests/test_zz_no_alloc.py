"""normalize_ragged_f32_noalloc: the ragged binary32 forward for callers that
must not allocate device memory (for instance code running under another
framework's memory pool, or a plugin whose host forbids allocation).  Its work
lists live in a fixed file-scope device array instead of a plan's cudaMalloc.

Checked here through the C ABI: two calls in a row, on different batches,
give the oracle's bits and the same bits as normalize_f32 with a plan; the
second call leaves the device's free memory unchanged; a vector with a
negative length is skipped (its outputs keep their fill values) while every
other vector still matches; a batch without elements (NULL x) finishes its
empty vectors; sizes beyond the fixed maximum are refused before any work.
This file is collected last on purpose."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_bits, cuda_device
from paper_1606_06508_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    dev = cuda_device()
    import __graft_entry__
    __graft_entry__.build()
    from paper_1606_06508_gb300 import _lib as L
    return torch, dev, L, torch.cuda.current_stream().cuda_stream


def _batch(count, seed, nmax):
    lengths = synth.ragged_lengths(count, seed=seed, nmax=nmax)
    lengths[::101] = 0
    lengths[3] = 5000
    off = synth.offsets_from_lengths(lengths)
    x = synth.ragged_values(lengths, np.float32, seed=seed)
    x[off[7]:off[8]] = 0
    return off, x


def _outputs(torch, dev, xt, count):
    y = torch.full_like(xt, float("nan"))
    r = torch.full((count,), float("nan"), device=dev)
    h = torch.full((count,), float("nan"), device=dev)
    c = torch.full((count,), 77, dtype=torch.int8, device=dev)
    return y, r, h, c


def _np(ts):
    return [t.cpu().numpy() for t in ts]


def _noalloc(L, xt, outs, count, ot, flags, stream):
    y, r, h, c = outs
    st = L.normalize_ragged_f32_noalloc(xt.data_ptr(), y.data_ptr(), r.data_ptr(), h.data_ptr(), c.data_ptr(),
                                        count, ot.data_ptr(), flags, stream)
    assert st == L.NGB_OK, L.last_error()


def _run(env, off, x):
    torch, dev, L, stream = env
    count = off.size - 1
    xt = torch.from_numpy(x).to(dev)
    ot = torch.from_numpy(off).to(dev)
    ref, mine = _outputs(torch, dev, xt, count), _outputs(torch, dev, xt, count)
    st, plan = L.ngb_plan_create(count, 4, 0)
    assert st == L.NGB_OK
    y, r, h, c = ref
    assert L.normalize_f32(xt.data_ptr(), y.data_ptr(), r.data_ptr(), h.data_ptr(), c.data_ptr(), count, 0,
                           ot.data_ptr(), plan, 0, stream) == L.NGB_OK
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    _noalloc(L, xt, mine, count, ot, 0, stream)
    torch.cuda.synchronize()
    free_after = torch.cuda.mem_get_info()[0]
    L.ngb_plan_destroy(plan)
    expect = oracle.normalize(x, dim=0, offsets=off)
    for a, b, o, what in zip(_np(mine), _np(ref), expect, ("y", "norm", "saved_h", "saved_code")):
        assert_bits(a, o, f"noalloc {what} vs oracle")
        assert_bits(a, b, f"noalloc {what} vs plan path")
    return free_before, free_after


def test_noalloc_matches_oracle_and_plan_path_twice(env):
    # first call (sets up the scratch address on this device), then a second,
    # different batch: the shared lists and counters must not leak between calls
    _run(env, *_batch(20011, seed=3, nmax=4096))
    fb, fa = _run(env, *_batch(7001, seed=8, nmax=2000))
    assert fa == fb, (fb, fa)


def test_noalloc_skips_a_vector_with_bad_offsets(env):
    """With NGB_VALIDATE_OFFSETS, vector 2 of this batch has a negative length:
    its norm, saved h and code keep their fill values; every other vector's
    per-vector outputs, and y of every vector no other vector overlaps, equal
    the oracle's (evaluated on the well-formed vectors) and the plan path's."""
    torch, dev, L, stream = env
    lengths = np.array([3, 5, 4, 7, 2, 9, 300, 1, 0, 40], dtype=np.int64)
    off = synth.offsets_from_lengths(lengths)
    x = synth.ragged_values(lengths, np.float32, seed=5)
    bad = off.copy()
    bad[2] = bad[3] + 1  # vector 2: negative length; vector 1 then overlaps vector 3
    count = lengths.size
    xt, ot = torch.from_numpy(x).to(dev), torch.from_numpy(bad).to(dev)
    mine = _outputs(torch, dev, xt, count)
    ref = _outputs(torch, dev, xt, count)
    _noalloc(L, xt, mine, count, ot, L.NGB_VALIDATE_OFFSETS, stream)
    from paper_1606_06508_gb300 import api
    plan = api.Plan(count, torch.float32)
    y, r, h, c = ref
    assert L.normalize_f32(xt.data_ptr(), y.data_ptr(), r.data_ptr(), h.data_ptr(), c.data_ptr(), count, 0,
                           ot.data_ptr(), plan.handle, L.NGB_VALIDATE_OFFSETS, stream) == L.NGB_OK
    assert plan.query_status() == L.NGB_ERR_BAD_OFFSETS
    plan.close()
    my, mr, mh, mc = _np(mine)
    ry, rr, rh, rc = _np(ref)
    assert np.isnan(mr[2]) and np.isnan(mh[2]) and mc[2] == 77
    ok = np.array([i != 2 for i in range(count)])
    # the oracle on each well-formed vector as the classifier reads it
    for i in np.flatnonzero(ok):
        s, e = int(bad[i]), int(bad[i + 1])
        oy, orr, oh, oc = oracle.normalize(x[s:e], dim=0, offsets=np.array([0, e - s], np.int64))
        assert_bits(mr[i:i + 1], orr, f"vector {i} norm")
        assert_bits(mh[i:i + 1], oh, f"vector {i} saved_h")
        assert_bits(mc[i:i + 1], oc, f"vector {i} code")
        if i not in (1, 3):  # vectors 1 and 3 overlap
            assert_bits(my[s:e], oy, f"vector {i} y")
    for a, b, what in ((mr, rr, "norm"), (mh, rh, "saved_h"), (mc, rc, "code")):
        assert_bits(a, b, f"{what} vs plan path")
    keep = np.ones(x.size, bool)
    keep[int(bad[1]):int(bad[4])] = False
    assert_bits(my[keep], ry[keep], "y vs plan path")


def test_noalloc_without_elements(env):
    """A batch of empty vectors passed with NULL x and y: norms +0, code zero."""
    torch, dev, L, stream = env
    count = 5
    ot = torch.zeros(count + 1, dtype=torch.int64, device=dev)
    r = torch.full((count,), float("nan"), device=dev)
    c = torch.full((count,), 77, dtype=torch.int8, device=dev)
    st = L.normalize_ragged_f32_noalloc(None, None, r.data_ptr(), None, c.data_ptr(), count, ot.data_ptr(), 0,
                                        stream)
    assert st == L.NGB_OK, L.last_error()
    rn, cn = _np((r, c))
    assert np.all(rn == 0) and not np.any(np.signbit(rn)) and np.all(cn == L.NGB_CODE_ZERO)


def test_noalloc_limits(env):
    _, _, L, _ = env
    big = L.NGB_NOALLOC_MAX_COUNT + 1
    assert L.normalize_ragged_f32_noalloc(8, 8, None, None, None, big, 8, 0, None) == L.NGB_ERR_UNSUPPORTED
    assert "NGB_NOALLOC_MAX_COUNT" in L.last_error()
    assert L.normalize_ragged_f32_noalloc(None, None, None, None, None, 0, None, 0, None) == L.NGB_OK
    assert L.normalize_ragged_f32_noalloc(None, None, None, None, None, 5, None, 0, None) == L.NGB_ERR_INVALID_ARG
    assert L.normalize_ragged_f32_noalloc(8, 8, None, None, None, 5, 8, 0x1, None) == L.NGB_ERR_INVALID_ARG
