"""The library's calls on pinned host memory (zero-copy): inputs and outputs
allocated with cudaHostAlloc (torch pin_memory) are passed to the C ABI as
they are, and the kernels read and write them over the host link.  Dense
binary32 quaternions, binary64 rows, a ragged binary32 batch (offsets in host
memory too) and a ragged binary64 backward, bit for bit against the oracle."""
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


def _pinned(torch, a):
    t = torch.empty(a.shape, dtype=torch.from_numpy(a[:0]).dtype, pin_memory=True)
    t.copy_(torch.from_numpy(a))
    return t


@pytest.mark.parametrize("f,dim,count", [("f32", 4, 300001), ("f64", 256, 3001), ("f64", 3, 10007)])
def test_dense_on_host_memory(env, f, dim, count):
    torch, dev, L, stream = env
    if dim == 4:
        x = synth.quaternions_f32(count, seed=21)
    elif dim == 3:
        x = synth.vectors3_f64(count, seed=22)
    else:
        x = synth.rows(count, dim, np.float64, seed=23)
    n_vec = x.shape[0]
    xh = _pinned(torch, x)
    yh = torch.empty_like(xh).pin_memory()
    rh = torch.empty(n_vec, dtype=xh.dtype).pin_memory()
    fn = L.normalize_f32 if f == "f32" else L.normalize_f64
    assert fn(xh.data_ptr(), yh.data_ptr(), rh.data_ptr(), None, None, n_vec, dim, None, None, 0, stream) == L.NGB_OK
    torch.cuda.synchronize()
    oy, orr, _, _ = oracle.normalize(x.reshape(-1), dim=dim)
    assert_bits(yh.numpy().reshape(-1), oy, f"{f} d={dim} y on host memory")
    assert_bits(rh.numpy(), orr, f"{f} d={dim} norm on host memory")


def test_ragged_forward_and_backward_on_host_memory(env):
    torch, dev, L, stream = env
    from paper_1606_06508_gb300 import api
    for f, dt in (("f32", np.float32), ("f64", np.float64)):
        lengths = synth.ragged_lengths(20011, seed=24, nmax=3000)
        lengths[::97] = 0
        off = synth.offsets_from_lengths(lengths)
        x = synth.ragged_values(lengths, dt, seed=24)
        g = synth.normal_like(x.shape, dt, seed=25)
        xh, offh, gh = _pinned(torch, x), _pinned(torch, off), _pinned(torch, g)
        yh, grh = torch.empty_like(xh).pin_memory(), torch.empty_like(xh).pin_memory()
        count = lengths.size
        td = xh.dtype
        h = torch.empty(count, dtype=td, device=dev)
        c = torch.empty(count, dtype=torch.int8, device=dev)
        plan = api.Plan(count, td)
        fwd = L.normalize_f32 if f == "f32" else L.normalize_f64
        bwd = L.normalize_backward_f32 if f == "f32" else L.normalize_backward_f64
        assert fwd(xh.data_ptr(), yh.data_ptr(), None, h.data_ptr(), c.data_ptr(), count, 0, offh.data_ptr(),
                   plan.handle, 0, stream) == L.NGB_OK
        assert bwd(yh.data_ptr(), gh.data_ptr(), h.data_ptr(), c.data_ptr(), grh.data_ptr(), count, 0, offh.data_ptr(),
                   plan.handle, 0, stream) == L.NGB_OK
        assert plan.query_status() == L.NGB_OK
        oy, _, oh, oc = oracle.normalize(x, dim=0, offsets=off)
        assert_bits(yh.numpy(), oy, f"ragged {f} y on host memory")
        assert_bits(h.cpu().numpy(), oh, f"ragged {f} saved_h")
        og = oracle.backward(oy, g, oh, oc, dim=0, offsets=off)
        assert_bits(grh.numpy(), og, f"ragged {f} grad on host memory")
        plan.close()
