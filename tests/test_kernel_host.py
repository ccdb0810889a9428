"""The kernels' per-thread arithmetic compiled for the host (csrc/ngb_arith.cuh
through tests/kernel_host_check.cpp, the CUDA intrinsics mapped to the host's
IEEE operations by tests/hostcuda/cuda_runtime.h) against the oracle, bit for
bit, on CPU: the n <= 4 forward in its integer-pipe and hardware forms, the
zero-padded form of the ragged thread items, the generic thread path for
5 <= n <= 16, the backward, the binary64 form with the squares on the FP64
pipe, and the quotient Algorithms 1 and 2.  The GPU parity tests check the same code on
the device; this catches a mistake in the arithmetic without one."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from gpu_util import assert_bits, f64_small_range_edges, full_grid_two_f32
from paper_1606_06508_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1606_06508_gb300", "csrc")
DT = {"f32": np.float32, "f64": np.float64}


@pytest.fixture(scope="module")
def khc(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("khc")
    exe = str(d / "kernel_host_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", os.path.join(HERE, "hostcuda"),
                    "-I", CSRC, os.path.join(HERE, "kernel_host_check.cpp"), "-o", exe], check=True)
    return exe, d


def _run(khc, f, dim, mode, quat_zero, parts):
    exe, d = khc
    src, dst = str(d / "in.bin"), str(d / "out.bin")
    with open(src, "wb") as fh:
        for p in parts:
            fh.write(np.ascontiguousarray(p).tobytes())
    subprocess.run([exe, f, str(dim), mode, "1" if quat_zero else "0", src, dst], check=True)
    return np.fromfile(dst, dtype=np.uint8)


def _forward(khc, x, dim, mode, flags=0):
    dt = x.dtype
    count = x.size // dim
    raw = _run(khc, "f32" if dt == np.float32 else "f64", dim, mode, not (flags & 1), [x.reshape(-1)])
    s = dt.itemsize
    y = raw[: count * dim * s].view(dt)
    r = raw[count * dim * s: (count * dim + count) * s].view(dt)
    h = raw[(count * dim + count) * s: (count * dim + 2 * count) * s].view(dt)
    c = raw[(count * dim + 2 * count) * s:].view(np.int8)
    return y, r, h, c


def _specials(x, rng):
    fi = np.finfo(x.dtype)
    vals = [0.0, -0.0, np.nan, np.inf, -np.inf, float(fi.max), float(fi.tiny), float(fi.smallest_subnormal),
            -3 * float(fi.smallest_subnormal), 1.0]
    cnt, n = x.shape
    for j in range(min(cnt // 4, 3000)):
        x[int(rng.integers(cnt)), int(rng.integers(n))] = vals[j % len(vals)]
    x[0] = 0
    x[1] = -0.0
    return x


def _check_forward(khc, x, dim, mode, flags=0, what=""):
    y, r, h, c = _forward(khc, x, dim, mode, flags)
    oy, orr, oh, oc = oracle.normalize(x.reshape(-1), dim=dim, flags=flags)
    assert_bits(y, oy, f"{what} y")
    assert_bits(r, orr, f"{what} norm")
    assert_bits(h, oh, f"{what} h")
    assert_bits(c, oc, f"{what} code")
    return oy, oh, oc


def _inputs(f, dim, seed):
    rng = np.random.default_rng(seed)
    if f == "f32":
        return [_specials(synth.vectors_f32(20000, dim, seed=seed), rng)]
    out = [_specials(synth.vectors_f64(20000, dim, seed=seed), rng),
           f64_small_range_edges(6000, dim, seed=seed) if dim <= 4 else None,
           np.ldexp(rng.uniform(1.0, 2.0, (20000, dim)) * np.where(rng.integers(0, 2, (20000, dim)) == 1, -1.0, 1.0),
                    rng.integers(-30, 31, (20000, dim)))]
    return [a for a in out if a is not None]


@pytest.mark.parametrize("f", ["f32", "f64"])
@pytest.mark.parametrize("dim", [1, 2, 3, 4])
def test_small_forward_matches_oracle(khc, f, dim):
    modes = ["fwd", "hw"] + (["padded", "sq64"] if f == "f64" else [])
    for k, x in enumerate(_inputs(f, dim, seed=40 + dim)):
        for mode in modes:  # ragged thread items keep the vector zero rule for n = 4
            _check_forward(khc, x, dim, mode, flags=1 if mode == "padded" else 0, what=f"{f} d={dim} set {k} {mode}")
        if dim == 4:
            _check_forward(khc, x, dim, "fwd", flags=1, what=f"{f} d=4 set {k} vector semantics")


def test_full_exponent_grid_two_components_f32(khc):
    """n = 2, binary32: every exponent pair in [-149, 127]^2, the mantissas
    {1, 1.5, 2 - 2^-23} for each component and the four sign patterns
    (2,762,244 vectors), bit for bit."""
    x = full_grid_two_f32(signs=(1.0, -1.0))
    x = np.concatenate([x, -x])
    assert x.shape == (4 * 277 * 277 * 9, 2)
    _check_forward(khc, x, 2, "fwd", what="f32 n=2 full exponent grid")


@pytest.mark.parametrize("f", ["f32", "f64"])
@pytest.mark.parametrize("alg", [1, 2])
def test_quotient_algorithms_match_oracle(khc, f, alg):
    """The quotient Algorithms 1 and 2 of the comparison kernels (y and r)."""
    rng = np.random.default_rng(alg)
    x = _specials(synth.vectors_f32(20000, 3, seed=alg) if f == "f32" else synth.vectors_f64(20000, 3, seed=alg), rng)
    y, r, _, _ = _forward(khc, x, 3, f"quot{alg}")
    oy, orr = oracle.quotient3(x, alg)
    assert_bits(y, oy.reshape(-1), f"{f} Algorithm {alg} y")
    assert_bits(r, orr, f"{f} Algorithm {alg} r")


def test_config0_vectors_take_the_integer_form(khc):
    """The 65,600 x 3 binary64 case through the library's forward."""
    x = synth.vectors3_f64(65536, seed=0)
    _check_forward(khc, x, 3, "fwd", what="65600 x 3 binary64")


@pytest.mark.parametrize("f", ["f32", "f64"])
@pytest.mark.parametrize("dim", [5, 7, 8, 13, 16])
def test_generic_thread_forward_matches_oracle(khc, f, dim):
    for k, x in enumerate(_inputs(f, dim, seed=60 + dim)):
        _check_forward(khc, x, dim, "fwd", what=f"{f} d={dim} set {k}")


@pytest.mark.parametrize("f", ["f32", "f64"])
@pytest.mark.parametrize("dim", [1, 2, 3, 4, 5, 9, 16])
def test_backward_matches_oracle(khc, f, dim):
    dt = DT[f]
    x = _inputs(f, dim, seed=80 + dim)[0]
    oy, _, oh, oc = oracle.normalize(x.reshape(-1), dim=dim)
    g = np.random.default_rng(dim).standard_normal(oy.size).astype(dt)
    raw = _run(khc, f, dim, "bwd", True, [oy, g, oh, oc.astype(np.int8)])
    og = oracle.backward(oy, g, oh, oc, dim=dim)
    assert_bits(raw.view(dt), og, f"{f} d={dim} grad")
