"""GPU parity of the quotient algorithms (Section 1, Algorithms 1 and 2) and
of the naive sequence (Table 4) with the oracle, bit for bit (NaN as a
class), through the C ABI."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_bits, cuda_device

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


def _vectors(dt, count, seed):
    rng = np.random.default_rng(seed)
    lo, hi, spread = (-100, 90, 30) if dt == np.float32 else (-900, 800, 200)
    base = rng.integers(lo, hi, size=(count, 1))
    e = base + rng.integers(-spread, spread + 1, size=(count, 3))
    x = np.ldexp(rng.uniform(1.0, 2.0, size=(count, 3)) * rng.choice([-1.0, 1.0], size=(count, 3)), e).astype(dt)
    x[: count // 4] = rng.standard_normal((count // 4, 3)).astype(dt)
    fi = np.finfo(dt)
    specials = [0.0, -0.0, np.nan, np.inf, -np.inf, float(fi.max), float(fi.tiny), float(fi.smallest_subnormal), 1.0]
    k = count // 4
    for j in range(min(count // 3, 3000)):
        x[k + j, j % 3] = specials[j % len(specials)]
        if j % 5 == 0:
            x[k + j, (j + 1) % 3] = specials[(j // 5) % len(specials)]
    x[0] = 0
    x[1] = (0, 0, -7)
    x[2] = (np.nan, 0, 0)
    x[3] = (0, np.nan, 0)
    x[4] = (5, 5, 5)          # ties between magnitudes
    x[5] = (-3, 3, 0)
    return x


@pytest.mark.parametrize("f", ["f32", "f64"])
@pytest.mark.parametrize("alg", [1, 2])
def test_quotient_parity(dev, f, alg):
    from paper_1606_06508_gb300 import api
    dt = DT[f]
    x = _vectors(dt, 20011, seed=alg)
    oy, orr = oracle.quotient3(x, alg)
    y, r = api.quotient_normalize3(_to(dev, x), alg, return_norm=True)
    assert_bits(_np(y), oy, f"{f} Algorithm {alg} y")
    assert_bits(_np(r), orr, f"{f} Algorithm {alg} r")
    xt = _to(dev, x)  # in place
    api.quotient_normalize3(xt, alg, out=xt)
    assert_bits(_np(xt), oy, f"{f} Algorithm {alg} in place")


@pytest.mark.parametrize("f", ["f32", "f64"])
@pytest.mark.parametrize("dim", [2, 3, 4])
def test_naive_parity(dev, f, dim):
    from paper_1606_06508_gb300 import api
    dt = DT[f]
    rng = np.random.default_rng(dim)
    x = rng.standard_normal((30001, dim)).astype(dt)
    x[:50] *= np.finfo(dt).max / 4     # overflows in the naive sequence
    x[50:100] *= np.finfo(dt).tiny      # underflows
    x[100] = 0
    y = api.naive_normalize(_to(dev, x))
    assert_bits(_np(y), oracle.naive(x, dim), f"{f} naive d={dim}")


def test_quotient_argument_errors(dev):
    import torch
    from paper_1606_06508_gb300 import _lib as L
    x = torch.zeros(10, 3, device=dev)
    st = L.quotient_normalize3_f32(x.data_ptr(), x.data_ptr(), None, 10, 3, None)
    assert st == L.NGB_ERR_INVALID_ARG
