"""Helpers for the GPU parity tests: bitwise comparison with NaN as a class."""
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
