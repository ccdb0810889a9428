"""The guard-padded buffers of tests/guarded.py on CPU tensors: writes inside
the array leave the guards intact, a write one element before or after it is
seen, and the array base moves off 16-byte alignment with `shift`."""
import numpy as np
import pytest
import torch

import host_args
from guarded import Guarded


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64, torch.int8])
@pytest.mark.parametrize("shift", [0, 1])
def test_guards_see_writes_outside_the_array(dtype, shift):
    g = Guarded(37, dtype, "cpu", shift=shift)
    g.fill(np.arange(37).astype(torch.empty(0, dtype=dtype).numpy().dtype))
    assert g.guards_intact()
    assert np.array_equal(g.values(), np.arange(37))
    g.view.fill_(3)
    assert g.guards_intact()
    g.buf[g.head + g.n] = 1  # one past the end
    assert not g.guards_intact()
    g2 = Guarded(5, dtype, "cpu", shift=shift)
    g2.buf[g2.head - 1] = 1  # one before the start
    assert not g2.guards_intact()


def test_shift_moves_the_base_off_16_bytes():
    for dtype in (torch.float32, torch.float64):
        a, b = Guarded(8, dtype, "cpu"), Guarded(8, dtype, "cpu", shift=1)
        assert (a.ptr() - a.buf.data_ptr()) % 16 == 0
        assert (b.ptr() - b.buf.data_ptr()) % 16 != 0


class _OracleStandIn:
    """The C ABI's forward and backward entry points over host pointers,
    answered by the oracle after the library's own argument checks
    (csrc/ngb_args.h built for the host, tests/host_args.py): a call the
    library rejects is rejected here with the same status, a ragged call needs
    a plan handle, and a ragged batch without an element array (NULL pointer)
    finishes its empty vectors and skips the others, as the library does.
    Exercises the guarded cases' buffers, pointers, sizes and checks on CPU
    tensors."""

    NGB_ERR_NO_PLAN = 5

    @staticmethod
    def _read(ptr, n, dt):
        import ctypes
        if n == 0:
            return np.zeros(0, dtype=dt)
        return np.frombuffer(ctypes.string_at(ptr, n * np.dtype(dt).itemsize), dtype=dt).copy()

    @staticmethod
    def _write(ptr, a, mask=None):
        import ctypes
        if ptr:
            a = np.ascontiguousarray(a)
            if mask is not None:
                old = _OracleStandIn._read(ptr, a.size, a.dtype)
                a = np.where(mask, a, old)
            ctypes.memmove(ptr, a.ctypes.data, a.nbytes)

    def _fwd(self, dt, xp, yp, rp, hp, cp, count, dim, offp, plan, flags, stream):
        import oracle
        st, no_elements = host_args.check_forward(xp, count, dim, offp, flags)
        if st != 0:
            return st
        if dim == 0 and not plan:
            return self.NGB_ERR_NO_PLAN
        if count == 0:
            return 0
        off = self._read(offp, count + 1, np.int64) if offp else None
        if no_elements:  # only the empty vectors are finished
            empty = np.diff(off) == 0
            _, r, h, c = oracle.normalize(np.zeros(0, dt), dim=0, offsets=np.zeros(count + 1, np.int64))
            for p, a in ((rp, r), (hp, h), (cp, c.astype(np.int8))):
                self._write(p, a, mask=empty)
            return 0
        n = int(off[-1]) if off is not None else count * dim
        y, r, h, c = oracle.normalize(self._read(xp, n, dt), dim=dim, offsets=off, flags=flags)
        for p, a in ((yp, y), (rp, r), (hp, h), (cp, c.astype(np.int8))):
            self._write(p, a)
        return 0

    def _bwd(self, dt, yp, gp, hp, cp, gradp, count, dim, offp, plan, flags, stream):
        import oracle
        st, no_elements = host_args.check_backward(yp, gp, hp, cp, gradp, count, dim, offp, flags)
        if st != 0:
            return st
        if dim == 0 and not plan:
            return self.NGB_ERR_NO_PLAN
        if count == 0 or no_elements:  # without elements there is nothing to write
            return 0
        off = self._read(offp, count + 1, np.int64) if offp else None
        n = int(off[-1]) if off is not None else count * dim
        grad = oracle.backward(self._read(yp, n, dt), self._read(gp, n, dt), self._read(hp, count, dt),
                               self._read(cp, count, np.int8), dim=dim, offsets=off)
        self._write(gradp, grad)
        return 0

    def normalize_f32(self, *a):
        return self._fwd(np.float32, *a)

    def normalize_f64(self, *a):
        return self._fwd(np.float64, *a)

    def normalize_backward_f32(self, *a):
        return self._bwd(np.float32, *a)

    def normalize_backward_f64(self, *a):
        return self._bwd(np.float64, *a)


FAKE_PLAN = 1  # a non-NULL plan handle for the stand-in's ragged calls


@pytest.mark.parametrize("f", ["f32", "f64"])
@pytest.mark.parametrize("shift", [0, 1])
def test_guarded_cases_run_on_cpu_with_the_oracle_standing_in(f, shift):
    """The dense cases and the ragged counts of tests/test_gpu_guards.py, among
    them a batch of one empty vector whose element buffers are NULL."""
    import guard_cases as gc
    from paper_1606_06508_gb300 import synth
    lib = _OracleStandIn()
    for dim, count in ((1, 3), (4, 33), (17, 2), (300, 3)):
        x = gc.dense_inputs(f, count, dim, seed=dim)
        fwd = gc.forward_case(lib, None, lambda: None, "cpu", f, x, count, dim, shift)
        gc.backward_case(lib, None, lambda: None, "cpu", f, fwd, count, dim, shift, seed=dim)
    for count in gc.RAGGED_COUNTS:
        lengths = gc.ragged_lengths_with_edges(count, seed=count)
        off = synth.offsets_from_lengths(lengths)
        x = synth.ragged_values(lengths, gc.NP[f], seed=count)
        fwd = gc.forward_case(lib, None, lambda: None, "cpu", f, x, count, 0, shift, offsets=off, plan=FAKE_PLAN)
        gc.backward_case(lib, None, lambda: None, "cpu", f, fwd, count, 0, shift, seed=count, offsets=off,
                         plan=FAKE_PLAN)


def test_stand_in_rejects_what_the_library_rejects():
    """The stand-in answers with the library's statuses: a dense call without x,
    a ragged call without a plan or offsets, a backward call without its saved
    state; a ragged call whose element arrays are NULL is accepted."""
    lib = _OracleStandIn()
    assert lib.normalize_f32(None, None, None, None, None, 3, 4, None, None, 0, None) == 1
    assert lib.normalize_f32(None, None, None, None, None, 3, 0, None, FAKE_PLAN, 0, None) == 1
    off = np.zeros(4, np.int64)
    assert lib.normalize_f32(None, None, None, None, None, 3, 0, off.ctypes.data, None, 0, None) == 5
    r = np.full(3, np.nan, np.float32)
    assert lib.normalize_f32(None, None, r.ctypes.data, None, None, 3, 0, off.ctypes.data, FAKE_PLAN, 0, None) == 0
    assert np.array_equal(r, np.zeros(3, np.float32))
    h = np.zeros(3, np.float32)
    assert lib.normalize_backward_f32(None, None, h.ctypes.data, None, None, 3, 0, off.ctypes.data, FAKE_PLAN, 0,
                                      None) == 1
