"""The warp and block forms of the kernels' arithmetic (csrc/ngb_rowpath.cuh:
rows in registers, half-warp rows, streaming warps, 4-row streaming batches,
streaming blocks, and their backward passes) compiled for the host and run
on an emulated block of threads (tests/hostwarp/cuda_runtime.h: warp
collectives and __syncthreads as barriers of std::threads), against the
oracle, bit for bit, on CPU.  The GPU parity tests check the same code on the
device; this checks the order CR(n), the streaming passes and the
integer-pipe binary64 steps without one."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from gpu_util import assert_bits, f64_range_edges
from paper_1606_06508_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1606_06508_gb300", "csrc")
DT = {"f32": np.float32, "f64": np.float64}


@pytest.fixture(scope="module")
def rph(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("rph")
    exe = str(d / "rowpath_host_check")
    r = subprocess.run([cxx, "-O2", "-std=c++20", "-ffp-contract=off", "-pthread", "-I",
                        os.path.join(HERE, "hostwarp"), "-I", CSRC, os.path.join(HERE, "rowpath_host_check.cpp"),
                        "-o", exe], capture_output=True, text=True)
    if r.returncode != 0 and "barrier" in r.stderr:
        pytest.skip("the host C++ library has no <barrier>")
    assert r.returncode == 0, r.stderr[-3000:]
    return exe, d


def _call(rph, f, n, path, parts):
    exe, d = rph
    src, dst = str(d / "in.bin"), str(d / "out.bin")
    with open(src, "wb") as fh:
        for p in parts:
            fh.write(np.ascontiguousarray(p).tobytes())
    subprocess.run([exe, f, str(n), path, src, dst], check=True, timeout=300)
    return np.fromfile(dst, dtype=np.uint8)


def _forward(rph, f, n, path, x, what):
    dt = DT[f]
    cnt, s = x.size // n, dt(0).itemsize
    raw = _call(rph, f, n, path, [x.reshape(-1)])
    y = raw[: cnt * n * s].view(dt)
    r = raw[cnt * n * s: (cnt * n + cnt) * s].view(dt)
    h = raw[(cnt * n + cnt) * s: (cnt * n + 2 * cnt) * s].view(dt)
    c = raw[(cnt * n + 2 * cnt) * s:].view(np.int8)
    oy, orr, oh, oc = oracle.normalize(x.reshape(-1), dim=n)
    assert_bits(y, oy, f"{what} y")
    assert_bits(r, orr, f"{what} norm")
    assert_bits(h, oh, f"{what} h")
    assert_bits(c, oc, f"{what} code")


def _backward(rph, f, n, path, x, what):
    dt = DT[f]
    oy, _, oh, oc = oracle.normalize(x.reshape(-1), dim=n)
    g = np.random.default_rng(n).standard_normal(oy.size).astype(dt)
    raw = _call(rph, f, n, path + "_bwd", [oy, g, oh, oc.astype(np.int8)])
    assert_bits(raw.view(dt), oracle.backward(oy, g, oh, oc, dim=n), f"{what} grad")


def _rows(f, cnt, n, seed):
    """Rows N(0,1) x 2^s (one s per row over most of the range), with zero
    rows, NaN, infinities, subnormals and the largest value planted."""
    dt = DT[f]
    x = synth.rows(cnt, n, dt, seed=seed)
    fi = np.finfo(dt)
    rng = np.random.default_rng(seed)
    if cnt > 6:
        x[1] = 0
        x[2, int(rng.integers(n))] = np.nan
        x[3, int(rng.integers(n))] = np.inf
        x[4] = 0
        x[4, int(rng.integers(n))] = fi.smallest_subnormal
        x[5, int(rng.integers(n))] = fi.max
        x[6, : n // 2] = fi.smallest_subnormal * rng.integers(1, 9, n // 2)
    return x


CASES = [  # (dtype, n, path, rows) following the library's dispatch of dense rows
    ("f32", 17, "warp", 13), ("f32", 33, "warp", 13), ("f32", 100, "warp", 13), ("f32", 255, "warp", 9),
    ("f32", 256, "warp", 9), ("f32", 257, "warp", 9), ("f32", 1000, "warp", 7), ("f32", 1024, "warp", 7),
    ("f32", 132, "half", 11), ("f32", 200, "half", 12), ("f32", 252, "half", 9), ("f32", 256, "half", 9),
    ("f32", 1025, "stream", 9), ("f32", 5000, "stream", 7), ("f32", 16385, "block", 7),
    ("f64", 17, "batch", 13), ("f64", 100, "batch", 11), ("f64", 256, "batch", 9), ("f64", 1000, "batch", 10),
    ("f64", 3000, "batch", 9), ("f64", 17, "stream", 9), ("f64", 300, "stream", 9), ("f64", 2048, "stream", 7),
    ("f64", 16385, "block", 7),
]


@pytest.mark.parametrize("f,n,path,cnt", CASES)
def test_rows_forward_matches_oracle(rph, f, n, path, cnt):
    _forward(rph, f, n, path, _rows(f, cnt, n, seed=n + cnt), f"{f} n={n} {path}")


@pytest.mark.parametrize("n,path", [(17, "batch"), (256, "batch"), (1000, "batch"), (40, "stream"),
                                    (3000, "stream"), (20000, "block")])
def test_f64_rows_integer_pipe_limits(rph, n, path):
    """binary64 rows whose smallest component sits on, below or above the
    limits of the integer-pipe steps."""
    x = f64_range_edges(max(9, min(30, 6000 // n)), n, seed=n)
    _forward(rph, "f64", n, path, x, f"f64 limits n={n} {path}")


@pytest.mark.parametrize("f,n,path", [("f32", 17, "warp"), ("f32", 100, "warp"), ("f32", 1024, "warp"),
                                      ("f32", 257, "warp"), ("f64", 33, "warp"), ("f64", 1000, "warp"),
                                      ("f32", 2048, "stream"), ("f64", 1025, "stream"), ("f64", 5000, "stream"),
                                      ("f32", 16385, "block"), ("f64", 16385, "block")])
def test_rows_backward_matches_oracle(rph, f, n, path):
    _backward(rph, f, n, path, _rows(f, 9, n, seed=3 * n), f"{f} n={n} {path}")


@pytest.mark.parametrize("n,path", [(40, "warp"), (1025, "stream"), (3000, "stream"), (17000, "block")])
def test_f64_backward_integer_pipe_limits(rph, n, path):
    x = f64_range_edges(12, n, seed=2 * n)
    _backward(rph, "f64", n, path, x, f"f64 limits n={n} {path}")


def test_grad_h_in_range_against_brute_force(rph):
    """grad_h_in_range (the binary64 backward's choice of f64emu::mul for
    d_k h and of f64emu::add_signed for d_k = RN(g_k - RN(y_k dot))) is never
    true for a row with a d_k outside mul()'s range or a g_k, p_k outside
    add_signed()'s.  Rows over the whole exponent range, with
    adversarial components: g_k = p_k (d_k = 0), g_k one ulp away from p_k
    (the smallest nonzero d_k), subnormal and huge g_k, zero y and dot, and
    rows whose d_k h sits on the upper limit."""
    n, cnt = 6, 40000
    rng = np.random.default_rng(11)
    sy = rng.integers(-1100, 1, size=(cnt, 1))
    y = rng.uniform(1, 2, size=(cnt, n)) * np.sign(rng.standard_normal((cnt, n))) * 2.0 ** sy
    y[rng.uniform(size=(cnt, n)) < 0.1] = 0.0
    dot = rng.uniform(1, 2, size=cnt) * np.sign(rng.standard_normal(cnt)) * 2.0 ** rng.integers(-1080, 1024, size=cnt)
    dot[::50] = 0.0
    g = rng.uniform(1, 2, size=(cnt, n)) * np.sign(rng.standard_normal((cnt, n))) * \
        2.0 ** rng.integers(-1100, 1023, size=(cnt, 1)) * 2.0 ** rng.integers(-40, 1, size=(cnt, n))
    with np.errstate(over="ignore", under="ignore"):
        p = y * dot[:, None]
        for i in range(cnt):
            k = int(rng.integers(n))
            kind = i % 4
            if kind == 0:
                g[i, k] = p[i, k]
            elif kind == 1:
                g[i, k] = np.nextafter(p[i, k], np.inf)
            elif kind == 2:
                g[i, k] = np.nextafter(p[i, k], -np.inf)
    h = rng.uniform(1, 2, size=cnt) * 2.0 ** rng.integers(-1022, 1024, size=cnt)
    g = np.where(np.isfinite(g), g, 0.0)
    # the upper edge: g_k near the top of binade E and p_k = y_k dot of the
    # opposite sign with its bound in binade E too, so that d_k reaches binade
    # E + 1; h puts E + 1 + e_h - 1023 just below, on and above 2045
    up = []
    for E in range(1030, 2041, 10):
        for eh in range(3064 - E, 3070 - E):
            yy = np.full(n, 2.0 ** -10)
            yy[0] = 1.99
            gg = np.full(n, 2.0 ** (E - 1023 - 30))
            gg[0] = 1.99 * 2.0 ** (E - 1023)
            up.append((yy, gg, -1.99 * 2.0 ** (E - 2 - 1023), 2.0 ** (eh - 1023)))
    # g_k in the top binade (exponent 2046), products by a small h in range:
    # add_signed's limit decides
    for eh in (1000, 990, 900):
        yy = np.full(n, 0.5)
        gg = np.full(n, 2.0 ** 1000)
        gg[1] = 1.5 * 2.0 ** 1023
        up.append((yy, gg, 0.75, 2.0 ** (eh - 1023)))
    y = np.concatenate([y, np.array([u[0] for u in up])])
    g = np.concatenate([g, np.array([u[1] for u in up])])
    dot = np.concatenate([dot, np.array([u[2] for u in up])])
    h = np.concatenate([h, np.array([u[3] for u in up])])
    cnt = dot.size
    raw = _call(rph, "f64", n, "ghr", [y.reshape(-1), g.reshape(-1), dot, h])
    decision, brute = raw[:cnt], raw[cnt:]
    taken = decision == 2
    assert not np.any(taken & (brute == 0)), np.flatnonzero(taken & (brute == 0))[:10]
    assert taken.sum() > cnt // 20 and (decision == 1).sum() > cnt // 20  # both answers occur
    tail = slice(cnt - len(up), cnt)  # the edge rows hold both answers of the brute force
    assert np.any(brute[tail] == 1) and np.any(brute[tail] == 0)


@pytest.mark.parametrize("n", [40, 300, 1025])
def test_f64_backward_product_by_h_over_the_exponent_range(rph, n):
    """The streaming binary64 backward (the ragged warp items) on inputs and
    upstream gradients over the whole exponent range, so that the products
    d_k h fall inside and outside f64emu::mul's range, row by row."""
    rng = np.random.default_rng(5 * n)
    cnt = 56
    sx = np.array([-1000, -600, -200, 0, 200, 600, 1000])
    sg = np.array([-1074, -1060, -1022, -1000, -900, -600, -300, 0, 300, 600, 900, 1000, 1015])
    x = rng.standard_normal((cnt, n)) * 2.0 ** sx[np.arange(cnt) % sx.size][:, None]
    oy, _, oh, oc = oracle.normalize(x.reshape(-1), dim=n)
    g = rng.standard_normal((cnt, n)) * 2.0 ** sg[(np.arange(cnt) * 5) % sg.size][:, None]
    g[::3, 0] = 2.0 ** 1000
    g[1::3, 1] = 5e-324
    g = g.reshape(-1)
    raw = _call(rph, "f64", n, "stream_bwd", [oy, g, oh, oc.astype(np.int8)])
    assert_bits(raw.view(np.float64), oracle.backward(oy, g, oh, oc, dim=n), f"f64 n={n} product by h")


def _group_lengths(cnt, n):
    return np.maximum(5, n - np.arange(cnt) % 5)


def _pack(rows2d, lengths):
    return np.concatenate([rows2d[i, :m] for i, m in enumerate(lengths)])


@pytest.mark.parametrize("f,n,w,cnt", [("f64", 64, 8, 37), ("f64", 9, 8, 21), ("f64", 128, 16, 23),
                                       ("f64", 65, 16, 19), ("f32", 64, 8, 29), ("f32", 128, 16, 19)])
def test_group_forward_and_backward_match_oracle(rph, f, n, w, cnt):
    """Groups of 8 or 16 lanes (csrc/ngb_grouppath.cuh), one vector each, the
    groups of a warp on vectors of different lengths and kinds (zero, NaN,
    infinite, subnormal components; scaled and unscaled), forward and
    backward; binary64 also at the limits of the integer-pipe steps."""
    dt = DT[f]
    sets = [_rows(f, cnt, n, seed=7 * n + w)]
    if f == "f64":
        sets.append(f64_range_edges(cnt, n, seed=n + w))
    for k, x in enumerate(sets):
        lengths = _group_lengths(x.shape[0], n)
        for i, m in enumerate(lengths):
            x[i, m:] = 0  # components past the vector's length are not part of it
        off = synth.offsets_from_lengths(lengths)
        xp = _pack(x, lengths)
        oy, orr, oh, oc = oracle.normalize(xp, dim=0, offsets=off)
        raw = _call(rph, f, n, f"group{w}", [x.reshape(-1)])
        c_ = x.shape[0]
        s_ = dt(0).itemsize
        y = raw[: c_ * n * s_].view(dt).reshape(c_, n)
        what = f"{f} n<={n} group{w} set {k}"
        assert_bits(_pack(y, lengths), oy, what + " y")
        assert_bits(raw[c_ * n * s_: (c_ * n + c_) * s_].view(dt), orr, what + " norm")
        assert_bits(raw[(c_ * n + c_) * s_: (c_ * n + 2 * c_) * s_].view(dt), oh, what + " h")
        assert_bits(raw[(c_ * n + 2 * c_) * s_:].view(np.int8), oc, what + " code")
        g = np.random.default_rng(n + k).standard_normal((c_, n)).astype(dt)
        yr = np.zeros((c_, n), dt)
        for i, m in enumerate(lengths):
            yr[i, :m] = oy[off[i]:off[i + 1]]
            g[i, m:] = 0
        og = oracle.backward(oy, _pack(g, lengths), oh, oc, dim=0, offsets=off)
        rawb = _call(rph, f, n, f"group{w}_bwd", [yr, g, oh, oc.astype(np.int8)])
        assert_bits(_pack(rawb.view(dt).reshape(c_, n), lengths), og, what + " grad")


@pytest.mark.parametrize("n,w", [(64, 8), (128, 16)])
def test_group_backward_product_by_h_over_the_exponent_range(rph, n, w):
    """binary64 group backward on inputs and upstream gradients over the whole
    exponent range (the products d_k h inside and outside f64emu::mul's
    range, group by group within a warp)."""
    rng = np.random.default_rng(3 * n + w)
    cnt = 56
    sx = np.array([-1000, -600, -200, 0, 200, 600, 1000])
    sg = np.array([-1074, -1060, -1022, -1000, -900, -600, -300, 0, 300, 600, 900, 1000, 1015])
    x = rng.standard_normal((cnt, n)) * 2.0 ** sx[np.arange(cnt) % sx.size][:, None]
    lengths = _group_lengths(cnt, n)
    for i, m in enumerate(lengths):
        x[i, m:] = 0
    off = synth.offsets_from_lengths(lengths)
    oy, _, oh, oc = oracle.normalize(_pack(x, lengths), dim=0, offsets=off)
    g = rng.standard_normal((cnt, n)) * 2.0 ** sg[(np.arange(cnt) * 5) % sg.size][:, None]
    g[::3, 0] = 2.0 ** 1000
    g[1::3, 1] = 5e-324
    yr = np.zeros((cnt, n))
    for i, m in enumerate(lengths):
        yr[i, :m] = oy[off[i]:off[i + 1]]
        g[i, m:] = 0
    og = oracle.backward(oy, _pack(g, lengths), oh, oc, dim=0, offsets=off)
    rawb = _call(rph, "f64", n, f"group{w}_bwd", [yr, g, oh, oc.astype(np.int8)])
    assert_bits(_pack(rawb.view(np.float64).reshape(cnt, n), lengths), og, f"f64 group{w} product by h")


@pytest.mark.parametrize("f,n", [("f64", 16), ("f64", 9), ("f32", 16)])
def test_thread_forward_matches_oracle(rph, f, n):
    """Thread items of the ragged forward (one thread per vector, lengths
    1 .. n): binary64 with the integer-pipe scale, squares and outputs, on
    vectors over the whole exponent range, at the limits of the integer-pipe
    steps (f64_range_edges), zero vectors, NaN and infinities."""
    dt = DT[f]
    cnt = 120
    lengths = 1 + np.arange(cnt) % n
    if f == "f64":
        x = np.concatenate([f64_range_edges(cnt // 2, n, seed=n), _rows(f, cnt - cnt // 2, n, seed=3 * n)])
    else:
        x = _rows(f, cnt, n, seed=3 * n)
    x[7] = 0
    x[13, 0] = np.inf
    x[19, -1] = np.nan
    x = x.astype(dt)
    for i, m in enumerate(lengths):
        x[i, m:] = 0
    off = synth.offsets_from_lengths(lengths)
    oy, orr, oh, oc = oracle.normalize(_pack(x, lengths), dim=0, offsets=off)
    raw = _call(rph, f, n, "thread", [x.reshape(-1)])
    s_ = dt(0).itemsize
    y = raw[: cnt * n * s_].view(dt).reshape(cnt, n)
    what = f"{f} thread forward n<={n}"
    assert_bits(_pack(y, lengths), oy, what + " y")
    assert_bits(raw[cnt * n * s_: (cnt * n + cnt) * s_].view(dt), orr, what + " norm")
    assert_bits(raw[(cnt * n + cnt) * s_: (cnt * n + 2 * cnt) * s_].view(dt), oh, what + " h")
    assert_bits(raw[(cnt * n + 2 * cnt) * s_:].view(np.int8), oc, what + " code")


@pytest.mark.parametrize("f,n", [("f64", 16), ("f64", 7), ("f32", 16)])
def test_thread_backward_over_the_exponent_range(rph, f, n):
    """Thread items of the ragged backward (one thread per vector, lengths 1
    .. n), binary64 with the integer-pipe products: inputs and upstream
    gradients over the whole exponent range, zero vectors and NaN, so that
    the products fall inside and outside f64emu's ranges vector by vector;
    every gradient against the oracle."""
    dt = DT[f]
    rng = np.random.default_rng(17 * n + len(f))
    cnt = 96
    lengths = 1 + np.arange(cnt) % n
    sx = np.array([-1000, -600, -200, 0, 200, 600, 1000]) if f == "f64" else np.array([-120, -60, 0, 60, 120])
    sg = (np.array([-1074, -1060, -1022, -1000, -900, -600, -300, 0, 300, 600, 900, 1000, 1015]) if f == "f64"
          else np.array([-149, -140, -126, -100, -50, 0, 50, 100, 120]))
    x = (rng.standard_normal((cnt, n)) * 2.0 ** sx[np.arange(cnt) % sx.size][:, None]).astype(dt)
    x[5] = 0
    x[11, 0] = np.nan
    for i, m in enumerate(lengths):
        x[i, m:] = 0
    off = synth.offsets_from_lengths(lengths)
    oy, _, oh, oc = oracle.normalize(_pack(x, lengths), dim=0, offsets=off)
    g = (rng.standard_normal((cnt, n)) * 2.0 ** sg[(np.arange(cnt) * 5) % sg.size][:, None]).astype(dt)
    g[::3, 0] = dt(2.0 ** (1000 if f == "f64" else 120))
    g[1::3, -1] = np.finfo(dt).smallest_subnormal
    yr = np.zeros((cnt, n), dt)
    for i, m in enumerate(lengths):
        yr[i, :m] = oy[off[i]:off[i + 1]]
        g[i, m:] = 0
    og = oracle.backward(oy, _pack(g, lengths), oh, oc, dim=0, offsets=off)
    rawb = _call(rph, f, n, "thread_bwd", [yr, g, oh, oc.astype(np.int8)])
    assert_bits(_pack(rawb.view(dt).reshape(cnt, n), lengths), og, f"{f} thread backward n<={n}")


@pytest.mark.parametrize("n", [1025, 5000])
def test_stream_speculation_falls_back(rph, n):
    """binary32 streaming rows whose first 256 components select another
    factor than the whole row (a larger component later): the speculative sum
    is dropped and the second pass gives the oracle's bits."""
    rng = np.random.default_rng(n)
    x = rng.standard_normal((6, n)).astype(np.float32)
    x[0, 700] = 2.0 ** 60          # first round: c = 1; row: sigma_max
    x[1, :256] *= 2.0 ** -80       # first round: sigma_min; row: c = 1
    x[2, :] *= 2.0 ** -80
    x[2, n - 1] = 2.0 ** 70        # first round: sigma_min; row: sigma_max
    x[3, :] *= 2.0 ** 60           # the whole row sigma_max (speculation holds)
    x[4, :256] = 0                 # first round all zero; row: c = 1
    _forward(rph, "f32", n, "stream", x, f"f32 n={n} speculation")


@pytest.mark.parametrize("f,n,cnt", [("f64", 300, 11), ("f64", 1000, 9), ("f64", 40, 13), ("f64", 20, 13),
                                     ("f64", 9, 11), ("f32", 700, 9)])
def test_pairs_forward_matches_oracle(rph, f, n, cnt):
    """Two vectors of different lengths per warp sharing one square root and
    reciprocal, with the partial-round skip (the ragged binary64 warp items),
    against the oracle; binary64 also at the integer-pipe limits."""
    dt = DT[f]
    sets = [_rows(f, cnt, n, seed=3 * n + cnt)]
    if f == "f64":
        sets.append(f64_range_edges(cnt, n, seed=n + 1))
    for k, x in enumerate(sets):
        lengths = _group_lengths(x.shape[0], n)
        for i, m in enumerate(lengths):
            x[i, m:] = 0
        off = synth.offsets_from_lengths(lengths)
        oy, orr, oh, oc = oracle.normalize(_pack(x, lengths), dim=0, offsets=off)
        raw = _call(rph, f, n, "pairs", [x.reshape(-1)])
        c_, s_ = x.shape[0], dt(0).itemsize
        what = f"{f} n<={n} pairs set {k}"
        assert_bits(_pack(raw[: c_ * n * s_].view(dt).reshape(c_, n), lengths), oy, what + " y")
        assert_bits(raw[c_ * n * s_: (c_ * n + c_) * s_].view(dt), orr, what + " norm")
        assert_bits(raw[(c_ * n + c_) * s_: (c_ * n + 2 * c_) * s_].view(dt), oh, what + " h")
        assert_bits(raw[(c_ * n + 2 * c_) * s_:].view(np.int8), oc, what + " code")
