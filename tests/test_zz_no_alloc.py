"""normalize_ragged_f32_noalloc: the ragged binary32 forward for callers that
must not allocate device memory (for instance code running under another
framework's memory pool, or a plugin whose host forbids allocation).  Its work
lists live in a fixed file-scope device array instead of a plan's cudaMalloc.

Checked here through the C ABI: two calls in a row, on different batches,
give the same bits as normalize_f32 with a plan; sizes beyond the fixed
maximum are refused before any work; the second call leaves the device's free
memory unchanged.  This file is collected last on purpose."""
import numpy as np
import pytest

from gpu_util import assert_bits, cuda_device
from paper_1606_06508_gb300 import synth

pytestmark = pytest.mark.gpu


def _batch(count, seed, nmax):
    lengths = synth.ragged_lengths(count, seed=seed, nmax=nmax)
    lengths[::101] = 0
    lengths[3] = 5000
    off = synth.offsets_from_lengths(lengths)
    x = synth.ragged_values(lengths, np.float32, seed=seed)
    x[off[7]:off[8]] = 0
    return off, x


def _run(L, torch, dev, off, x, stream):
    count = off.size - 1
    xt = torch.from_numpy(x).to(dev)
    ot = torch.from_numpy(off).to(dev)
    outs = {}
    for name in ("ref", "noalloc"):
        y = torch.full_like(xt, float("nan"))
        r = torch.empty(count, device=dev)
        h = torch.empty(count, device=dev)
        c = torch.empty(count, dtype=torch.int8, device=dev)
        outs[name] = (y, r, h, c)
    st, plan = L.ngb_plan_create(count, 4, 0)
    assert st == L.NGB_OK
    y, r, h, c = outs["ref"]
    assert L.normalize_f32(xt.data_ptr(), y.data_ptr(), r.data_ptr(), h.data_ptr(), c.data_ptr(), count, 0,
                           ot.data_ptr(), plan, 0, stream) == L.NGB_OK
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    y, r, h, c = outs["noalloc"]
    st = L.normalize_ragged_f32_noalloc(xt.data_ptr(), y.data_ptr(), r.data_ptr(), h.data_ptr(), c.data_ptr(),
                                        count, ot.data_ptr(), 0, stream)
    assert st == L.NGB_OK, L.last_error()
    torch.cuda.synchronize()
    free_after = torch.cuda.mem_get_info()[0]
    L.ngb_plan_destroy(plan)
    for a, b, what in zip(outs["noalloc"], outs["ref"], ("y", "norm", "saved_h", "saved_code")):
        assert_bits(a.cpu().numpy(), b.cpu().numpy(), f"noalloc {what}")
    return free_before, free_after


def test_noalloc_matches_plan_path_twice():
    import torch
    dev = cuda_device()
    import __graft_entry__
    __graft_entry__.build()
    from paper_1606_06508_gb300 import _lib as L
    stream = torch.cuda.current_stream().cuda_stream
    # first call (sets up the scratch address on this device), then a second,
    # different batch: the shared lists and counters must not leak between calls
    _run(L, torch, dev, *_batch(20011, seed=3, nmax=4096), stream)
    fb, fa = _run(L, torch, dev, *_batch(7001, seed=8, nmax=2000), stream)
    assert fa == fb, (fb, fa)


def test_noalloc_limits():
    cuda_device()
    import __graft_entry__
    __graft_entry__.build()
    from paper_1606_06508_gb300 import _lib as L
    big = L.NGB_NOALLOC_MAX_COUNT + 1
    assert L.normalize_ragged_f32_noalloc(8, 8, None, None, None, big, 8, 0, None) == L.NGB_ERR_UNSUPPORTED
    assert "NGB_NOALLOC_MAX_COUNT" in L.last_error()
    assert L.normalize_ragged_f32_noalloc(None, None, None, None, None, 0, None, 0, None) == L.NGB_OK
    assert L.normalize_ragged_f32_noalloc(None, None, None, None, None, 5, None, 0, None) == L.NGB_ERR_INVALID_ARG
