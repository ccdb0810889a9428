"""Splitting a batch across ranks (one process per GPU).  Every vector is
independent, so a batch shards into contiguous vector ranges with no
exchange between ranks: dense batches by vector count, ragged batches
balanced by element count through the offsets."""
from __future__ import annotations

import numpy as np


def dense_range(count: int, world: int, rank: int) -> tuple[int, int]:
    """Vectors [a, b) of rank `rank` out of `world` for a dense batch."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    return (count * rank) // world, (count * (rank + 1)) // world


def ragged_range(offsets, world: int, rank: int) -> tuple[int, int]:
    """Vectors [a, b) of rank `rank` for a ragged batch: the boundaries are the
    first vectors starting at or after rank * total / world elements."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    off = np.asarray(offsets, dtype=np.int64)
    count = off.size - 1
    total = int(off[-1] - off[0])

    def cut(r):
        if r <= 0:
            return 0
        if r >= world:
            return count
        target = off[0] + (total * r) // world
        return int(np.searchsorted(off[:-1], target, side="left"))

    return cut(rank), cut(rank + 1)
