"""torch-facing helpers over the C ABI: they take torch CUDA tensors, pass their
data pointers, sizes and the current CUDA stream to the entry points of
libnormgb, and return torch tensors.  torch provides device memory and
streams only; every step of the normalization runs in the library's kernels.

    y = normalize(x)                       # dense [..., d]
    y, r = normalize(x, return_norm=True)
    y = normalize(values, offsets=off)     # ragged, int64 offsets [count + 1]
    y = NormalizeFn.apply(x)               # differentiable (hand-written backward)
    R = normalize_to_rotation(q)           # [count, 3, 3]
"""
from __future__ import annotations

import torch

from . import _lib as L

_FLOAT = {torch.float32: ("f32", 4), torch.float64: ("f64", 8)}


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def _ptr(t):
    return None if t is None else t.data_ptr()


def _check_tensor(t, name, dtype=None):
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor (there is no CPU path)")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must have dtype {dtype}, not {t.dtype}")


def _sfx(dtype):
    if dtype not in _FLOAT:
        raise TypeError(f"only float32 and float64 are supported, not {dtype}")
    return _FLOAT[dtype]


class Plan:
    """A ragged-batch plan (work lists, mapping, CUDA graphs) for `count`
    vectors of one dtype, on the current device.  Mirrors ngb_plan_*."""

    def __init__(self, count: int, dtype=torch.float32, capacity: int = 0):
        _, nbytes = _sfx(dtype)
        st, h = L.ngb_plan_create(count, nbytes, capacity)
        L.check(st, "ngb_plan_create")
        self.handle = h
        self.count = count
        self.dtype = dtype

    def close(self):
        if getattr(self, "handle", None):
            L.ngb_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_mapping(self, thread_max=8, warp_max=8192, block_threads=256, grid_blocks=0):
        L.check(L.ngb_plan_set_mapping(self.handle, thread_max, warp_max, block_threads, grid_blocks),
                "ngb_plan_set_mapping")

    @property
    def mapping(self):
        st, m = L.ngb_plan_get_mapping(self.handle)
        L.check(st, "ngb_plan_get_mapping")
        return m

    def autotune(self, offsets: torch.Tensor, cache_path: str | None = None):
        _check_tensor(offsets, "offsets", torch.int64)
        st = L.ngb_plan_autotune(self.handle, offsets.data_ptr(),
                                 cache_path.encode() if cache_path else None, _stream())
        L.check(st, "ngb_plan_autotune")
        return self.mapping

    def set_graphs(self, enable: bool):
        L.check(L.ngb_plan_set_graphs(self.handle, 1 if enable else 0), "ngb_plan_set_graphs")

    def query_status(self) -> int:
        """Synchronizes and returns the raw status (NGB_OK or NGB_ERR_BAD_OFFSETS)."""
        return L.ngb_query_status(self.handle, _stream())


_plans: dict = {}


def plan_for(count: int, dtype, device=None) -> Plan:
    """A cached default plan per (device, count, dtype)."""
    dev = torch.cuda.current_device() if device is None else device
    key = (dev, count, dtype)
    p = _plans.get(key)
    if p is None:
        p = _plans[key] = Plan(count, dtype)
    return p


def normalize(x: torch.Tensor, offsets: torch.Tensor | None = None, *, out: torch.Tensor | None = None,
              return_norm: bool = False, save: bool = False, vector_semantics: bool = False,
              validate_offsets: bool = False, plan: Plan | None = None, norm_only: bool = False):
    """Normalize the vectors of x.

    Dense: x has shape [..., d]; every row of the last dimension is a vector.
    Ragged: x is 1-D packed values and offsets an int64 CUDA tensor [count + 1].
    Returns y (or None with norm_only), plus norm if return_norm, plus
    (saved_h, saved_code) if save.
    """
    _check_tensor(x, "x")
    sfx, _ = _sfx(x.dtype)
    if offsets is None:
        if x.dim() < 1:
            raise ValueError("x must have at least one dimension")
        dim = x.shape[-1]
        count = x.numel() // dim if dim > 0 else 0
        off_ptr = None
        plan_h = None
    else:
        _check_tensor(offsets, "offsets", torch.int64)
        dim = 0
        count = offsets.numel() - 1
        off_ptr = offsets.data_ptr()
        if plan is None:
            plan = plan_for(count, x.dtype)
        plan_h = plan.handle
    y = None
    if not norm_only:
        y = torch.empty_like(x) if out is None else out
        _check_tensor(y, "out", x.dtype)
    norm = torch.empty(count, dtype=x.dtype, device=x.device) if (return_norm or norm_only) else None
    h = torch.empty(count, dtype=x.dtype, device=x.device) if save else None
    code = torch.empty(count, dtype=torch.int8, device=x.device) if save else None
    flags = (L.NGB_VECTOR_SEMANTICS if vector_semantics else 0) | (L.NGB_VALIDATE_OFFSETS if validate_offsets else 0)
    fn = L.normalize_f32 if sfx == "f32" else L.normalize_f64
    st = fn(x.data_ptr(), _ptr(y), _ptr(norm), _ptr(h), _ptr(code), count, dim, off_ptr, plan_h, flags, _stream())
    L.check(st, f"normalize_{sfx}")
    res = []
    if not norm_only:
        res.append(y)
    if return_norm or norm_only:
        res.append(norm)
    if save:
        res.extend([h, code])
    return res[0] if len(res) == 1 else tuple(res)


def normalize_backward(y, g, saved_h, saved_code, offsets=None, *, out=None, plan: Plan | None = None):
    """grad = (g - y (y.g)) / |x| from the forward's y, saved_h and saved_code."""
    for t, n in ((y, "y"), (g, "g"), (saved_h, "saved_h")):
        _check_tensor(t, n, y.dtype)
    _check_tensor(saved_code, "saved_code", torch.int8)
    sfx, _ = _sfx(y.dtype)
    if offsets is None:
        dim = y.shape[-1]
        count = y.numel() // dim if dim > 0 else 0
        off_ptr, plan_h = None, None
    else:
        _check_tensor(offsets, "offsets", torch.int64)
        dim, count, off_ptr = 0, offsets.numel() - 1, offsets.data_ptr()
        if plan is None:
            plan = plan_for(count, y.dtype)
        plan_h = plan.handle
    grad = torch.empty_like(g) if out is None else out
    fn = L.normalize_backward_f32 if sfx == "f32" else L.normalize_backward_f64
    st = fn(y.data_ptr(), g.data_ptr(), saved_h.data_ptr(), saved_code.data_ptr(), grad.data_ptr(), count, dim,
            off_ptr, plan_h, 0, _stream())
    L.check(st, f"normalize_backward_{sfx}")
    return grad


class NormalizeFn(torch.autograd.Function):
    """y = x/|x| with the scaling algorithms, differentiable: the forward saves
    y, h = 1/r~ and the factor code; the backward kernel reads y, g and the
    saved state once (x is not read again).

    It always uses the vector zero rule (NGB_VECTOR_SEMANTICS): a dense
    four-component zero input gives y = 0, not the quaternion (0, 0, 1, 0)
    that normalize() returns without the flag.  Either zero result is a
    constant, and the gradient at a zero input is +0."""

    @staticmethod
    def forward(ctx, x, offsets=None, plan=None):
        y, h, code = normalize(x.contiguous(), offsets, save=True, vector_semantics=True, plan=plan)
        ctx.save_for_backward(y, h, code, offsets if offsets is not None else torch.empty(0))
        ctx.ragged = offsets is not None
        ctx.plan = plan
        return y

    @staticmethod
    def backward(ctx, g):
        y, h, code, off = ctx.saved_tensors
        grad = normalize_backward(y, g.contiguous(), h, code, off if ctx.ragged else None, plan=ctx.plan)
        return grad, None, None


def normalize_to_rotation(q: torch.Tensor, return_norm: bool = False):
    """Quaternions [count, 4] (scalar part last) -> rotation matrices [count, 3, 3]."""
    _check_tensor(q, "q")
    sfx, _ = _sfx(q.dtype)
    if q.shape[-1] != 4:
        raise ValueError("quaternions have 4 components")
    count = q.numel() // 4
    R = torch.empty(q.shape[:-1] + (3, 3), dtype=q.dtype, device=q.device)
    norm = torch.empty(count, dtype=q.dtype, device=q.device) if return_norm else None
    fn = L.normalize_to_rotation_f32 if sfx == "f32" else L.normalize_to_rotation_f64
    L.check(fn(q.data_ptr(), R.data_ptr(), _ptr(norm), count, _stream()), f"normalize_to_rotation_{sfx}")
    return (R, norm) if return_norm else R


def copy_(dst: torch.Tensor, src: torch.Tensor):
    """Measurement aid: device copy through the library's streaming kernel."""
    _check_tensor(dst, "dst")
    _check_tensor(src, "src")
    nbytes = src.numel() * src.element_size()
    if dst.numel() * dst.element_size() < nbytes:
        raise ValueError("dst too small")
    L.check(L.ngb_copy(dst.data_ptr(), src.data_ptr(), nbytes, _stream()), "ngb_copy")
    return dst


def naive_normalize(x: torch.Tensor, out: torch.Tensor | None = None):
    """Measurement aid: y = x / sqrt(sum x^2) without scaling (Table 4's naive algorithm)."""
    _check_tensor(x, "x")
    sfx, _ = _sfx(x.dtype)
    dim = x.shape[-1]
    y = torch.empty_like(x) if out is None else out
    fn = L.naive_normalize_f32 if sfx == "f32" else L.naive_normalize_f64
    L.check(fn(x.data_ptr(), y.data_ptr(), x.numel() // dim, dim, _stream()), f"naive_normalize_{sfx}")
    return y


def quotient_normalize3(x: torch.Tensor, alg: int, out: torch.Tensor | None = None, return_norm: bool = False):
    """The paper's quotient Algorithm 1 or 2 (Section 1) on vectors [..., 3]."""
    _check_tensor(x, "x")
    sfx, _ = _sfx(x.dtype)
    if x.shape[-1] != 3:
        raise ValueError("the quotient algorithms take three components")
    count = x.numel() // 3
    y = torch.empty_like(x) if out is None else out
    norm = torch.empty(count, dtype=x.dtype, device=x.device) if return_norm else None
    fn = L.quotient_normalize3_f32 if sfx == "f32" else L.quotient_normalize3_f64
    L.check(fn(x.data_ptr(), y.data_ptr(), _ptr(norm), count, alg, _stream()), f"quotient_normalize3_{sfx}")
    return (y, norm) if return_norm else y
