"""The library's argument checks (csrc/ngb_args.h) built for the host through
tests/args_host_check.cpp into a small shared library, loaded with ctypes.
CPU tests use it to accept and reject calls exactly as the C ABI does."""
import ctypes
import os
import shutil
import subprocess
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1606_06508_gb300", "csrc")
INCLUDE = os.path.join(ROOT, "include")

_lib = None


def load():
    global _lib
    if _lib is None:
        cxx = shutil.which("g++") or shutil.which("c++")
        if cxx is None:
            raise RuntimeError("no C++ compiler for the host argument checks")
        out = os.path.join(tempfile.mkdtemp(prefix="ngb_args_"), "libargs.so")
        subprocess.run([cxx, "-O1", "-std=c++17", "-shared", "-fPIC", "-I", CSRC, "-I", INCLUDE,
                        os.path.join(HERE, "args_host_check.cpp"), "-o", out], check=True)
        L = ctypes.CDLL(out)
        P, I64, I32, U32, IP = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32, \
            ctypes.POINTER(ctypes.c_int)
        L.host_check_forward.argtypes = [P, I64, I32, P, U32, IP]
        L.host_check_backward.argtypes = [P, P, P, P, P, I64, I32, P, U32, IP]
        L.host_check_noalloc.argtypes = [P, I64, P, U32, IP]
        for f in (L.host_check_forward, L.host_check_backward, L.host_check_noalloc):
            f.restype = ctypes.c_int
        _lib = L
    return _lib


def _call(fn, *args):
    ne = ctypes.c_int(0)
    st = fn(*args, ctypes.byref(ne))
    return st, bool(ne.value)


def check_forward(x, count, dim, offsets, flags):
    """(status, no_elements) of normalize_f32/_f64's argument checks."""
    return _call(load().host_check_forward, x, count, dim, offsets, flags)


def check_backward(y, g, saved_h, saved_code, grad, count, dim, offsets, flags):
    """(status, no_elements) of normalize_backward_f32/_f64's argument checks."""
    return _call(load().host_check_backward, y, g, saved_h, saved_code, grad, count, dim, offsets, flags)


def check_noalloc(x, count, offsets, flags):
    """(status, no_elements) of normalize_ragged_f32_noalloc's argument checks."""
    return _call(load().host_check_noalloc, x, count, offsets, flags)
