"""ctypes binding of libnormgb (include/normgb.h).  Argument marshalling only:
every function below forwards its arguments to the C entry point of the same
name, which runs the CUDA kernels.  Pointers are Python ints (device
addresses), streams are cudaStream_t handles as ints (0 = legacy default).

The library is loaded on first use from this package's directory; if it is
missing or fails to load, an ImportError is raised: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnormgb.so")

NGB_OK = 0
NGB_ERR_INVALID_ARG = 1
NGB_ERR_UNSUPPORTED = 2
NGB_ERR_BAD_OFFSETS = 3
NGB_ERR_CUDA = 4
NGB_ERR_NO_PLAN = 5
STATUS_NAMES = {0: "NGB_OK", 1: "NGB_ERR_INVALID_ARG", 2: "NGB_ERR_UNSUPPORTED", 3: "NGB_ERR_BAD_OFFSETS",
                4: "NGB_ERR_CUDA", 5: "NGB_ERR_NO_PLAN"}

NGB_VECTOR_SEMANTICS = 0x1
NGB_VALIDATE_OFFSETS = 0x2
NGB_CODE_ONE, NGB_CODE_SIGMA_MIN, NGB_CODE_SIGMA_MAX, NGB_CODE_ZERO = 0, 1, 2, 3
NGB_MAX_LEN = 1 << 20

P = ctypes.c_void_p
I64 = ctypes.c_int64
I32 = ctypes.c_int32
U32 = ctypes.c_uint32
ST = ctypes.c_int

# name -> (restype, argtypes), in the order of include/normgb.h
PROTOTYPES = {
    "normalize_f32": (ST, [P, P, P, P, P, I64, I32, P, P, U32, P]),
    "normalize_f64": (ST, [P, P, P, P, P, I64, I32, P, P, U32, P]),
    "normalize_backward_f32": (ST, [P, P, P, P, P, I64, I32, P, P, U32, P]),
    "normalize_backward_f64": (ST, [P, P, P, P, P, I64, I32, P, P, U32, P]),
    "ngb_plan_create": (ST, [ctypes.POINTER(P), I64, I32, I64]),
    "ngb_plan_destroy": (ST, [P]),
    "ngb_plan_set_mapping": (ST, [P, I32, I32, I32, I32]),
    "ngb_plan_get_mapping": (ST, [P, ctypes.POINTER(I32), ctypes.POINTER(I32), ctypes.POINTER(I32),
                                  ctypes.POINTER(I32)]),
    "ngb_plan_autotune": (ST, [P, P, ctypes.c_char_p, P]),
    "ngb_plan_set_graphs": (ST, [P, I32]),
    "ngb_query_status": (ST, [P, P]),
    "ngb_quat_bulk_state": (ST, [ctypes.POINTER(U32)]),
    "normalize_to_rotation_f32": (ST, [P, P, P, I64, P]),
    "normalize_to_rotation_f64": (ST, [P, P, P, I64, P]),
    "ngb_copy": (ST, [P, P, I64, P]),
    "ngb_fp64_probe": (ST, [P, I32, I32, P, P]),
    "quotient_normalize3_f32": (ST, [P, P, P, I64, I32, P]),
    "quotient_normalize3_f64": (ST, [P, P, P, I64, I32, P]),
    "naive_normalize_f32": (ST, [P, P, I64, I32, P]),
    "naive_normalize_f64": (ST, [P, P, I64, I32, P]),
    "ngb_shard_range": (ST, [P, I64, I32, I32, ctypes.POINTER(I64), ctypes.POINTER(I64)]),
    "normalize_ragged_f32_noalloc": (ST, [P, P, P, P, P, I64, P, U32, P]),
    "ngb_last_error": (ctypes.c_char_p, []),
    "ngb_version": (ctypes.c_char_p, []),
}

_lib = None
_lock = threading.Lock()


class NormgbError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def lib():
    """The loaded library (ImportError if it is missing: build it with build.py)."""
    global _lib
    if _lib is None:
        with _lock:
            if _lib is None:
                if not os.path.exists(LIB_PATH):
                    raise ImportError(f"libnormgb.so not found at {LIB_PATH}; run "
                                      "`python -c 'import __graft_entry__ as g; g.build()'` first")
                L = ctypes.CDLL(LIB_PATH)
                for name, (res, args) in PROTOTYPES.items():
                    f = getattr(L, name)
                    f.restype = res
                    f.argtypes = args
                _lib = L
    return _lib


def check(status: int, where: str) -> None:
    if status != NGB_OK:
        raise NormgbError(status, where, last_error())


def last_error() -> str:
    return lib().ngb_last_error().decode()


def version() -> str:
    return lib().ngb_version().decode()


def _fwd(name):
    def f(*args):
        return getattr(lib(), name)(*args)
    f.__name__ = name
    f.__doc__ = f"C entry point {name} of include/normgb.h (raw status returned)."
    return f


normalize_f32 = _fwd("normalize_f32")
normalize_f64 = _fwd("normalize_f64")
normalize_backward_f32 = _fwd("normalize_backward_f32")
normalize_backward_f64 = _fwd("normalize_backward_f64")
ngb_plan_destroy = _fwd("ngb_plan_destroy")
ngb_plan_set_mapping = _fwd("ngb_plan_set_mapping")
ngb_plan_autotune = _fwd("ngb_plan_autotune")
ngb_plan_set_graphs = _fwd("ngb_plan_set_graphs")
ngb_query_status = _fwd("ngb_query_status")
normalize_to_rotation_f32 = _fwd("normalize_to_rotation_f32")
normalize_to_rotation_f64 = _fwd("normalize_to_rotation_f64")
ngb_copy = _fwd("ngb_copy")
ngb_fp64_probe = _fwd("ngb_fp64_probe")
quotient_normalize3_f32 = _fwd("quotient_normalize3_f32")
quotient_normalize3_f64 = _fwd("quotient_normalize3_f64")
naive_normalize_f32 = _fwd("naive_normalize_f32")
naive_normalize_f64 = _fwd("naive_normalize_f64")
normalize_ragged_f32_noalloc = _fwd("normalize_ragged_f32_noalloc")
NGB_NOALLOC_MAX_COUNT = 262144


def ngb_plan_create(count: int, dtype_bytes: int, capacity: int = 0):
    """Returns (status, plan handle as int or None)."""
    h = P()
    st = lib().ngb_plan_create(ctypes.byref(h), count, dtype_bytes, capacity)
    return st, h.value


def ngb_shard_range(offsets_ptr, count: int, world: int, rank: int):
    """Returns (status, begin, end); offsets_ptr is a host address or None."""
    b, e = I64(), I64()
    st = lib().ngb_shard_range(offsets_ptr, count, world, rank, ctypes.byref(b), ctypes.byref(e))
    return st, b.value, e.value


def ngb_plan_get_mapping(plan):
    a, b, c, d = I32(), I32(), I32(), I32()
    st = lib().ngb_plan_get_mapping(plan, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d))
    return st, (a.value, b.value, c.value, d.value)
