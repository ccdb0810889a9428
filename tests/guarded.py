"""Guard-padded buffers for out-of-bounds write checks, the stand-in for a
memory checker: each array sits between two guard zones filled with a known
byte pattern, and after a call both zones must still hold it."""
import numpy as np
import torch

GUARD_BYTES = 512
PATTERN = 0xA5


class Guarded:
    """n elements of `dtype` inside a torch buffer on `device` with GUARD_BYTES
    of guard on each side; `shift` extra elements before the array move its
    base off a 16-byte boundary (for 4- and 8-byte elements)."""

    def __init__(self, n, dtype, device, shift=0):
        self.itemsize = torch.empty(0, dtype=dtype).element_size()
        self.head = GUARD_BYTES // self.itemsize + shift
        self.n = n
        self.buf = torch.empty(self.head + n + GUARD_BYTES // self.itemsize, dtype=dtype, device=device)
        self.buf.view(torch.uint8).fill_(PATTERN)
        self.view = self.buf[self.head:self.head + n]

    def fill(self, values):
        """Copy `values` (numpy, n elements) into the array."""
        self.view.copy_(torch.from_numpy(np.ascontiguousarray(values).reshape(-1)))
        return self

    def ptr(self):
        return self.view.data_ptr()

    def guards_intact(self):
        b = self.buf.view(torch.uint8).cpu().numpy()
        head = b[: self.head * self.itemsize]
        tail = b[(self.head + self.n) * self.itemsize:]
        return bool(np.all(head == PATTERN) and np.all(tail == PATTERN))

    def values(self):
        return self.view.cpu().numpy()
