"""Column shards for one process per GPU.

Vertical columns are independent of one another within an implicit stage
(Sec. 3, the vertical problem decouples column by column; Sec. 4.3), so a
multi-GPU run partitions the global column set into contiguous ranges, one
per rank, and needs no data-path collective: each rank sets up its own
context over its range and steps it.  The only cross-rank traffic is
host-side bookkeeping (a barrier and a max over ranks of the timed region).

Shards are balanced by per-column work, not by column count, so that a mix of
size classes (different Nez, N) still gives every rank about the same load.
The default weight of a column is the size of its band factor, ldab * n with
ldab = 3k + 1 and k = 3(N + 1) - 1 (Sec. 4.3, the banded LU of the
vertically implicit operator): factor bytes, solve traffic and refinement
work all scale with it.
"""

from __future__ import annotations

from typing import Sequence

import numpy as np


def column_work(class_of_col, classes: Sequence[tuple[int, int]]) -> np.ndarray:
    """Weight of each column: ldab * n of its size class (nez, N)."""
    cls = np.asarray(class_of_col, dtype=np.int64)
    w = np.empty(len(classes), dtype=np.float64)
    for c, (nez, N) in enumerate(classes):
        n = 3 * (nez * N + 1)
        k = 3 * (N + 1) - 1
        w[c] = float((3 * k + 1) * n)
    if cls.size and (cls.min() < 0 or cls.max() >= len(classes)):
        raise ValueError("class id out of range")
    return w[cls]


def column_shards(ncols: int, world: int, weights=None) -> list[tuple[int, int]]:
    """Split columns [0, ncols) into `world` contiguous ranges [start, stop).

    Without weights the ranges differ in length by at most one column.  With
    weights (one non-negative value per column) shard r ends at the first
    column whose running weight reaches (r + 1) / world of the total, so each
    shard's weight exceeds total / world by less than one column's weight.
    Shards may be empty when world > ncols.
    """
    if world < 1:
        raise ValueError("world must be >= 1")
    if ncols < 0:
        raise ValueError("ncols must be >= 0")
    if weights is None:
        bounds = [(r * ncols) // world for r in range(world + 1)]
    else:
        w = np.asarray(weights, dtype=np.float64)
        if w.shape != (ncols,):
            raise ValueError("weights must have one entry per column")
        if ncols and (not np.all(np.isfinite(w)) or w.min() < 0):
            raise ValueError("weights must be finite and non-negative")
        cum = np.concatenate([[0.0], np.cumsum(w)])
        total = cum[-1]
        if total <= 0:
            return column_shards(ncols, world)
        targets = total * np.arange(1, world, dtype=np.float64) / world
        inner = np.searchsorted(cum, targets, side="left")
        bounds = [0] + [int(min(max(b, 0), ncols)) for b in inner] + [ncols]
        for r in range(1, world + 1):  # monotone even under rounding
            bounds[r] = max(bounds[r], bounds[r - 1])
    return [(int(bounds[r]), int(bounds[r + 1])) for r in range(world)]


def shard_of(ncols: int, rank: int, world: int, weights=None) -> tuple[int, int]:
    """This rank's [start, stop) of `column_shards`."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    return column_shards(ncols, world, weights)[rank]
