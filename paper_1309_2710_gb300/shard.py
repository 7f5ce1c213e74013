"""Splitting independent cells (or whole instances) across GPUs.

Cells of an operator-split flow step are independent (Section 2.1), so a
multi-GPU run needs no exchange during integration: each rank integrates its
own contiguous block of cells, or its own set of instances, and the results
are concatenated. These helpers choose the blocks; nothing here touches
device data.
"""
from __future__ import annotations

from typing import List, Optional, Sequence, Tuple

import numpy as np


def shard_cells(total: int, world: int, rank: int,
                weights: Optional[Sequence[float]] = None) -> Tuple[int, int]:
    """[start, stop) of rank's contiguous block of `total` cells. With
    per-cell weights (e.g. the previous flow step's f evaluations) the blocks
    carry about equal total weight; otherwise equal cell counts."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    if weights is None:
        base, extra = divmod(total, world)
        start = rank * base + min(rank, extra)
        return start, start + base + (1 if rank < extra else 0)
    w = np.asarray(weights, dtype=np.float64)
    if w.shape != (total,) or (w < 0).any():
        raise ValueError("weights must be non-negative, one per cell")
    c = np.concatenate([[0.0], np.cumsum(w)])
    targets = c[-1] * np.arange(world + 1) / world
    cuts = np.searchsorted(c, targets, side="left")
    cuts[0], cuts[-1] = 0, total
    cuts = np.maximum.accumulate(np.minimum(cuts, total))
    return int(cuts[rank]), int(cuts[rank + 1])


def shard_instances(sizes: Sequence[int], world: int) -> List[List[int]]:
    """Whole instances per rank, longest first onto the least loaded rank."""
    loads = [0] * world
    out: List[List[int]] = [[] for _ in range(world)]
    for i in sorted(range(len(sizes)), key=lambda i: -sizes[i]):
        r = min(range(world), key=lambda r: loads[r])
        out[r].append(i)
        loads[r] += sizes[i]
    return [sorted(x) for x in out]
