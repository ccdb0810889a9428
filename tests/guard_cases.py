"""Cases of the guard-padded checks (tests/test_gpu_guards.py): every input and
output of one C-ABI call sits in a Guarded buffer; after the call every guard
must be intact and every output bit-identical to the oracle.  `lib` is the
library's ctypes handle on the GPU; the CPU test of this module passes a
stand-in that writes the oracle's results through the same pointers."""
import numpy as np
import torch

import oracle
from guarded import Guarded
from gpu_util import assert_bits
from paper_1606_06508_gb300 import synth

NP = {"f32": np.float32, "f64": np.float64}
RAGGED_COUNTS = (1, 2, 19, 40, 257)  # count 1 is one empty vector: its element buffers are NULL
TD = {"f32": torch.float32, "f64": torch.float64}


def dense_inputs(f, count, dim, seed):
    """The wide-exponent recipe (with zeros, subnormals) for short vectors, the
    rows recipe (N(0,1) x 2^s per row) for long ones."""
    if dim <= 16:
        x = synth.vectors_f32(count, dim, seed=seed) if f == "f32" else synth.vectors_f64(count, dim, seed=seed)
        if count > 2:
            x[1] = 0
        return x
    return synth.rows(count, dim, NP[f], seed=seed)


def _check_guards(bufs):
    for name, g in bufs.items():
        assert g.guards_intact(), f"the guard of {name} was overwritten"


def forward_case(lib, stream, sync, device, f, x, count, dim, shift, offsets=None, plan=None, flags=0):
    """One forward call on guarded buffers; returns the oracle's (y, r, h, code)."""
    td = TD[f]
    n = x.size
    bufs = {"x": Guarded(n, td, device, shift).fill(x), "y": Guarded(n, td, device, shift),
            "norm": Guarded(count, td, device, shift), "saved_h": Guarded(count, td, device, shift),
            "saved_code": Guarded(count, torch.int8, device, shift)}
    off = None
    if offsets is not None:
        bufs["offsets"] = off = Guarded(count + 1, torch.int64, device, 0).fill(offsets)
    fn = lib.normalize_f32 if f == "f32" else lib.normalize_f64
    st = fn(bufs["x"].ptr(), bufs["y"].ptr(), bufs["norm"].ptr(), bufs["saved_h"].ptr(), bufs["saved_code"].ptr(),
            count, dim, off.ptr() if off is not None else None, plan, flags, stream)
    assert st == 0, st
    sync()
    _check_guards(bufs)
    o = oracle.normalize(x.reshape(-1), dim=dim, offsets=offsets, flags=flags)
    tag = f"{f} dim={dim} count={count} shift={shift}"
    for name, ref in zip(("y", "norm", "saved_h", "saved_code"), o):
        assert_bits(bufs[name].values(), ref, f"{tag} {name}")
    return o


def backward_case(lib, stream, sync, device, f, fwd, count, dim, shift, seed, offsets=None, plan=None):
    """One backward call on guarded buffers from the forward's (y, r, h, code)."""
    td = TD[f]
    oy, _, oh, oc = fwd
    g = np.random.default_rng(seed).standard_normal(oy.size).astype(NP[f])
    bufs = {"y": Guarded(oy.size, td, device, shift).fill(oy), "g": Guarded(oy.size, td, device, shift).fill(g),
            "saved_h": Guarded(count, td, device, shift).fill(oh),
            "saved_code": Guarded(count, torch.int8, device, shift).fill(oc.astype(np.int8)),
            "grad": Guarded(oy.size, td, device, shift)}
    off = None
    if offsets is not None:
        bufs["offsets"] = off = Guarded(count + 1, torch.int64, device, 0).fill(offsets)
    fn = lib.normalize_backward_f32 if f == "f32" else lib.normalize_backward_f64
    st = fn(bufs["y"].ptr(), bufs["g"].ptr(), bufs["saved_h"].ptr(), bufs["saved_code"].ptr(), bufs["grad"].ptr(),
            count, dim, off.ptr() if off is not None else None, plan, 0, stream)
    assert st == 0, st
    sync()
    _check_guards(bufs)
    og = oracle.backward(oy, g, oh, oc, dim=dim, offsets=offsets)
    assert_bits(bufs["grad"].values(), og, f"{f} dim={dim} count={count} shift={shift} grad")


def ragged_lengths_with_edges(count, seed):
    """Lengths 0 to 9000: empty and length-1 vectors, every length of the
    thread items, warp items, and one vector above the warp items' limit."""
    rng = np.random.default_rng(seed)
    lengths = rng.integers(0, 40, size=count).astype(np.int64)
    lengths[: min(count, 18)] = np.arange(min(count, 18))
    if count > 20:
        lengths[20] = 9000
        lengths[-1] = 257
    return lengths
