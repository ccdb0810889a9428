"""Splitting a batch across ranks (one process per GPU).  Every vector is
independent, so a batch shards into contiguous vector ranges with no
exchange between ranks: dense batches by vector count, ragged batches
balanced by element count through the offsets.  The ranges come from the
library's ngb_shard_range (include/normgb.h); this module passes host arrays
to it."""
from __future__ import annotations

import numpy as np

from . import _lib as L


def dense_range(count: int, world: int, rank: int) -> tuple[int, int]:
    """Vectors [a, b) of rank `rank` out of `world` for a dense batch."""
    st, a, b = L.ngb_shard_range(None, int(count), int(world), int(rank))
    if st != L.NGB_OK:
        raise ValueError(f"ngb_shard_range: {L.last_error()}")
    return a, b


def ragged_range(offsets, world: int, rank: int) -> tuple[int, int]:
    """Vectors [a, b) of rank `rank` for a ragged batch (host int64 offsets
    [count + 1]): the boundaries are the first vectors starting at or after
    offsets[0] + rank * total / world elements."""
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    st, a, b = L.ngb_shard_range(off.ctypes.data, off.size - 1, int(world), int(rank))
    if st != L.NGB_OK:
        raise ValueError(f"ngb_shard_range: {L.last_error()}")
    return a, b
