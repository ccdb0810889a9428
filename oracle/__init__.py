"""The oracle: a plain single-threaded C implementation of the paper's scaling
algorithms (Mascarenhas, arXiv 1606.06508, Section 2, Algorithms 3-7), loaded
with ctypes.

TEST INFRASTRUCTURE ONLY.  It may be imported by the tests, by the smoke check
and by the CPU-baseline leg of the benchmark, never by the library.  It shares
no code with the CUDA path.

``build()`` compiles ``normalize_oracle.c`` with gcc, ``-O2 -ffp-contract=off
-fno-fast-math`` (one IEEE operation per source operation, no fused
multiply-add), into ``liboracle.so`` beside this file.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "normalize_oracle.c")
HDR = os.path.join(HERE, "oracle_impl.h")
LIB = os.path.join(HERE, "liboracle.so")
# A prebuilt oracle library to load instead (the mutation test of the pins
# points this at deliberately broken copies); never built here.
LIB_OVERRIDE = os.environ.get("NGB_ORACLE_LIB")

CODE_ONE, CODE_SMIN, CODE_SMAX, CODE_ZERO = 0, 1, 2, 3
VECTOR_SEMANTICS = 1
CR_SLOTS = 256
MAX_LEN = 1 << 20

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fno-unsafe-math-optimizations",
          "-fPIC", "-shared", "-Wall", "-Wextra"]

_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the oracle library if it is missing or older than its sources."""
    if LIB_OVERRIDE:
        return LIB_OVERRIDE
    stale = (not os.path.exists(LIB) or
             os.path.getmtime(LIB) < max(os.path.getmtime(SRC), os.path.getmtime(HDR)))
    if force or stale:
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", *CFLAGS, SRC, "-o", tmp, "-lm"], check=True)
        os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            for sfx in ("f32", "f64"):
                f = getattr(lib, f"oracle_normalize_{sfx}")
                f.restype = ctypes.c_int
                f.argtypes = [P, ctypes.c_int64, ctypes.c_int32, P, ctypes.c_uint32, P, P, P, P]
                b = getattr(lib, f"oracle_backward_{sfx}")
                b.restype = ctypes.c_int
                b.argtypes = [P, P, P, P, ctypes.c_int64, ctypes.c_int32, P, P]
                rot = getattr(lib, f"oracle_rotation_{sfx}")
                rot.restype = ctypes.c_int
                rot.argtypes = [P, ctypes.c_int64, P, P]
                qt = getattr(lib, f"oracle_quotient3_{sfx}")
                qt.restype = ctypes.c_int
                qt.argtypes = [P, ctypes.c_int64, ctypes.c_int, P, P]
                nv = getattr(lib, f"oracle_naive_{sfx}")
                nv.restype = ctypes.c_int
                nv.argtypes = [P, ctypes.c_int64, ctypes.c_int32, P]
            lib.oracle_ieee_check.restype = ctypes.c_int
            lib.oracle_ieee_check.argtypes = []
            _lib = lib
    return _lib


def ieee_check() -> bool:
    """True when the compiled oracle rounds each operation separately and keeps subnormals."""
    return bool(_load().oracle_ieee_check())


def _ptr(a):
    return None if a is None else a.ctypes.data


def _sfx(dtype) -> str:
    dtype = np.dtype(dtype)
    if dtype == np.float32:
        return "f32"
    if dtype == np.float64:
        return "f64"
    raise TypeError(f"oracle supports float32 and float64, not {dtype}")


def normalize(x, dim: int = 0, offsets=None, flags: int = 0, count: int | None = None):
    """Normalize a dense ``[count][dim]`` batch (``dim > 0``) or a ragged batch
    (``dim == 0``, int64 ``offsets`` of length count+1).

    Returns ``(y, norm, saved_h, saved_code)`` as numpy arrays: y has x's
    shape (flattened layout kept), norm and saved_h one value per vector, and
    saved_code the int8 factor code (0: c = 1, 1: sigma_min, 2: sigma_max,
    3: zero input)."""
    x = np.ascontiguousarray(x)
    sfx = _sfx(x.dtype)
    if dim > 0:
        n_vec = x.size // dim if count is None else count
        off = None
    else:
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        n_vec = off.size - 1
    y = np.empty_like(x)
    norm = np.empty(n_vec, dtype=x.dtype)
    h = np.empty(n_vec, dtype=x.dtype)
    code = np.empty(n_vec, dtype=np.int8)
    rc = getattr(_load(), f"oracle_normalize_{sfx}")(
        _ptr(x), n_vec, dim, _ptr(off), flags, _ptr(y), _ptr(norm), _ptr(h), _ptr(code))
    if rc != 0:
        raise ValueError(f"oracle_normalize_{sfx} failed with code {rc}")
    return y, norm, h, code


def backward(y, g, saved_h, saved_code, dim: int = 0, offsets=None):
    """grad = ((g - y (y.g)) * h) * c per vector, for the outputs of :func:`normalize`."""
    y = np.ascontiguousarray(y)
    g = np.ascontiguousarray(g, dtype=y.dtype)
    saved_h = np.ascontiguousarray(saved_h, dtype=y.dtype)
    saved_code = np.ascontiguousarray(saved_code, dtype=np.int8)
    sfx = _sfx(y.dtype)
    off = None if dim > 0 else np.ascontiguousarray(offsets, dtype=np.int64)
    n_vec = saved_h.size
    grad = np.empty_like(y)
    rc = getattr(_load(), f"oracle_backward_{sfx}")(
        _ptr(y), _ptr(g), _ptr(saved_h), _ptr(saved_code), n_vec, dim, _ptr(off), _ptr(grad))
    if rc != 0:
        raise ValueError(f"oracle_backward_{sfx} failed with code {rc}")
    return grad


def normalize_threads(x, dim: int, offsets=None, flags: int = 0, threads: int = 1):
    """:func:`normalize` run over contiguous vector ranges on ``threads`` host
    threads (ctypes releases the GIL during each call).  Same results."""
    x = np.ascontiguousarray(x)
    if dim > 0:
        n_vec = x.size // dim
    else:
        offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        n_vec = offsets.size - 1
    y = np.empty_like(x)
    norm = np.empty(n_vec, dtype=x.dtype)
    h = np.empty(n_vec, dtype=x.dtype)
    code = np.empty(n_vec, dtype=np.int8)
    sfx = _sfx(x.dtype)
    fn = getattr(_load(), f"oracle_normalize_{sfx}")
    bounds = np.linspace(0, n_vec, threads + 1).astype(np.int64)
    isz = x.itemsize
    errors = []

    def work(a, b):
        if b <= a:
            return
        if dim > 0:
            xs = x.ctypes.data + int(a) * dim * isz
            ys = y.ctypes.data + int(a) * dim * isz
            offp = None
        else:
            # a ragged slice keeps absolute offsets: shift the base pointers back
            xs = x.ctypes.data
            ys = y.ctypes.data
            offp = offsets.ctypes.data + int(a) * 8
        rc = fn(xs, int(b - a), dim, offp, flags, ys, norm.ctypes.data + int(a) * isz,
                h.ctypes.data + int(a) * isz, code.ctypes.data + int(a))
        if rc:
            errors.append(rc)

    ts = [threading.Thread(target=work, args=(bounds[i], bounds[i + 1])) for i in range(threads)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    if errors:
        raise ValueError(f"oracle failed: {errors}")
    return y, norm, h, code


def backward_threads(y, g, saved_h, saved_code, dim: int = 0, offsets=None, threads: int = 1):
    """:func:`backward` run over contiguous vector ranges on ``threads`` host
    threads (ctypes releases the GIL during each call).  Same results."""
    y = np.ascontiguousarray(y)
    g = np.ascontiguousarray(g, dtype=y.dtype)
    saved_h = np.ascontiguousarray(saved_h, dtype=y.dtype)
    saved_code = np.ascontiguousarray(saved_code, dtype=np.int8)
    off = None if dim > 0 else np.ascontiguousarray(offsets, dtype=np.int64)
    n_vec = saved_h.size
    grad = np.empty_like(y)
    fn = getattr(_load(), f"oracle_backward_{_sfx(y.dtype)}")
    bounds = np.linspace(0, n_vec, threads + 1).astype(np.int64)
    isz = y.itemsize
    errors = []

    def work(a, b):
        if b <= a:
            return
        if dim > 0:
            shift = int(a) * dim * isz
            offp = None
        else:  # absolute offsets: keep the base pointers, move the offsets
            shift = 0
            offp = off.ctypes.data + int(a) * 8
        rc = fn(y.ctypes.data + shift, g.ctypes.data + shift, saved_h.ctypes.data + int(a) * isz,
                saved_code.ctypes.data + int(a), int(b - a), dim, offp, grad.ctypes.data + shift)
        if rc:
            errors.append(rc)

    ts = [threading.Thread(target=work, args=(bounds[i], bounds[i + 1])) for i in range(threads)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    if errors:
        raise ValueError(f"oracle failed: {errors}")
    return grad


def rotation(q):
    """Section 4: rotation matrices [count, 3, 3] of quaternions [count, 4]
    (scalar part last) normalized by Algorithm 7, and their norms."""
    q = np.ascontiguousarray(q)
    sfx = _sfx(q.dtype)
    count = q.size // 4
    R = np.empty((count, 3, 3), dtype=q.dtype)
    norm = np.empty(count, dtype=q.dtype)
    rc = getattr(_load(), f"oracle_rotation_{sfx}")(_ptr(q), count, _ptr(R), _ptr(norm))
    if rc != 0:
        raise ValueError(f"oracle_rotation_{sfx} failed with code {rc}")
    return R, norm


def quotient3(x, alg: int):
    """The paper's quotient Algorithm 1 or 2 (Section 1) on vectors [count, 3]:
    (y [count, 3], r [count])."""
    x = np.ascontiguousarray(x)
    sfx = _sfx(x.dtype)
    count = x.size // 3
    y = np.empty_like(x)
    norm = np.empty(count, dtype=x.dtype)
    rc = getattr(_load(), f"oracle_quotient3_{sfx}")(_ptr(x), count, int(alg), _ptr(y), _ptr(norm))
    if rc != 0:
        raise ValueError(f"oracle_quotient3_{sfx} failed with code {rc}")
    return y, norm


def naive(x, dim: int):
    """The unscaled sequence of Table 4: y = x * (1 / sqrt(sum x_k^2)) on [count, dim]."""
    x = np.ascontiguousarray(x)
    sfx = _sfx(x.dtype)
    count = x.size // dim
    y = np.empty_like(x)
    rc = getattr(_load(), f"oracle_naive_{sfx}")(_ptr(x), count, int(dim), _ptr(y))
    if rc != 0:
        raise ValueError(f"oracle_naive_{sfx} failed with code {rc}")
    return y
