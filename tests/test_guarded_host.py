"""The guard-padded buffers of tests/guarded.py on CPU tensors: writes inside
the array leave the guards intact, a write one element before or after it is
seen, and the array base moves off 16-byte alignment with `shift`."""
import numpy as np
import pytest
import torch

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
    answered by the oracle: exercises the guarded cases' buffers, pointers,
    sizes and checks on CPU tensors."""

    @staticmethod
    def _read(ptr, n, dt):
        import ctypes
        return np.frombuffer(ctypes.string_at(ptr, n * np.dtype(dt).itemsize), dtype=dt).copy()

    @staticmethod
    def _write(ptr, a):
        import ctypes
        if ptr:
            a = np.ascontiguousarray(a)
            ctypes.memmove(ptr, a.ctypes.data, a.nbytes)

    def _fwd(self, dt, xp, yp, rp, hp, cp, count, dim, offp, plan, flags, stream):
        import oracle
        off = self._read(offp, count + 1, np.int64) if offp else None
        n = int(off[-1]) if off is not None else count * dim
        y, r, h, c = oracle.normalize(self._read(xp, n, dt), dim=dim, offsets=off, flags=flags)
        for p, a in ((yp, y), (rp, r), (hp, h), (cp, c.astype(np.int8))):
            self._write(p, a)
        return 0

    def _bwd(self, dt, yp, gp, hp, cp, gradp, count, dim, offp, plan, flags, stream):
        import oracle
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


@pytest.mark.parametrize("f", ["f32", "f64"])
@pytest.mark.parametrize("shift", [0, 1])
def test_guarded_cases_run_on_cpu_with_the_oracle_standing_in(f, shift):
    import guard_cases as gc
    from paper_1606_06508_gb300 import synth
    lib = _OracleStandIn()
    for dim, count in ((1, 3), (4, 33), (17, 2), (300, 3)):
        x = gc.dense_inputs(f, count, dim, seed=dim)
        fwd = gc.forward_case(lib, None, lambda: None, "cpu", f, x, count, dim, shift)
        gc.backward_case(lib, None, lambda: None, "cpu", f, fwd, count, dim, shift, seed=dim)
    lengths = gc.ragged_lengths_with_edges(40, seed=1)
    off = synth.offsets_from_lengths(lengths)
    x = synth.ragged_values(lengths, gc.NP[f], seed=1)
    fwd = gc.forward_case(lib, None, lambda: None, "cpu", f, x, len(lengths), 0, shift, offsets=off)
    gc.backward_case(lib, None, lambda: None, "cpu", f, fwd, len(lengths), 0, shift, seed=2, offsets=off)
