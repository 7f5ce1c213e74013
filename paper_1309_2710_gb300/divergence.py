"""The warp divergence measure D of Section 3.1.

For a warp of 32 threads, thread i integrating one cell with d_i evaluations
of f (summed over one or more global time steps),

    D = sum_i d_i / (32 max_i d_i) .

D = 1 when every thread does the same work; D = 1/32 when one thread does
all of it. The paper uses D on its thread-per-ODE mapping, where thread i of
warp w integrates cell 32 w + i in the order the cells are stored; it reports
the distribution of D over 2048 warps (65,536 cells, ten global steps) for
"similar" (consecutive ignition samples) and "random" (shuffled) orderings.

Two readings where the paper is silent:
- a final partial warp of n < 32 cells uses n in the denominator (its idle
  lanes are not counted as work units);
- a warp whose cells did no f evaluations at all has D = 1.

A fixed mapping runs warp w for max_i d_i evaluations, so the share of lane
slots that do work over all warps is the lane efficiency
E = sum_i d_i / (32 sum_w max_{i in w} d_i). Sorting the cells by count and
cutting consecutive warps minimises sum_w max_w (the k-th largest warp
maximum is at least the ((k-1) 32 + 1)-th largest count, and the sorted cut
reaches that bound), so it is the best E any fixed mapping of the same cells
can reach.

The lane-per-cell kernels here do not keep a cell in a fixed warp slot (a
lane that finishes takes the next cell of a cost-sorted queue), so D over
the storage order says what the paper's fixed mapping would see, and D over
the cells sorted by their counts is what the best fixed mapping would see.
Host-side analysis of the per-cell statistics; nothing here touches device
data.
"""
from __future__ import annotations

from typing import Dict, Sequence

import numpy as np

WARP = 32


def warp_D(d: Sequence[int], width: int = WARP) -> np.ndarray:
    """D of every consecutive group of `width` cells of d (per-cell f-evaluation
    counts, in the order they map onto threads)."""
    d = np.asarray(d, dtype=np.float64).ravel()
    if width < 1:
        raise ValueError("width must be positive")
    if (d < 0).any():
        raise ValueError("f-evaluation counts are non-negative")
    n = d.shape[0]
    if n == 0:
        return np.zeros(0)
    groups = -(-n // width)
    pad = groups * width - n
    dp = np.concatenate([d, np.zeros(pad)]).reshape(groups, width)
    sizes = np.full(groups, float(width))
    if pad:
        sizes[-1] = width - pad
    mx = dp.max(axis=1)
    out = np.ones(groups)
    busy = mx > 0
    out[busy] = dp[busy].sum(axis=1) / (sizes[busy] * mx[busy])
    return out


def histogram(D: np.ndarray, bins: int = 20) -> np.ndarray:
    """Counts of D over `bins` equal bins of [0, 1] (D = 1 falls in the last)."""
    return np.histogram(np.asarray(D, dtype=np.float64), bins=bins, range=(0.0, 1.0))[0]


def lane_efficiency(d: Sequence[int], width: int = WARP) -> float:
    """E = sum d / (width sum_w max_w) for consecutive groups of `width` (a
    partial last warp still occupies a full warp slot); 1 for no work."""
    d = np.asarray(d, dtype=np.float64).ravel()
    if d.size == 0:
        return 1.0
    groups = -(-d.size // width)
    dp = np.concatenate([d, np.zeros(groups * width - d.size)]).reshape(groups, width)
    tot = dp.max(axis=1).sum()
    return float(d.sum() / (width * tot)) if tot > 0 else 1.0


def summary(d: Sequence[int], width: int = WARP, bins: int = 20) -> Dict[str, object]:
    """D statistics and lane efficiency of d in its given order and of d
    sorted by count (the best fixed mapping of the same cells)."""
    d = np.asarray(d).ravel()
    ds = np.sort(d)[::-1]

    def stats(x, e):
        if x.size == 0:
            return {"warps": 0, "lane_efficiency": e}
        return {"warps": int(x.size), "mean": float(x.mean()),
                "p10": float(np.percentile(x, 10)), "p50": float(np.percentile(x, 50)),
                "p90": float(np.percentile(x, 90)), "lane_efficiency": e,
                "hist": histogram(x, bins).tolist()}

    return {"given_order": stats(warp_D(d, width), lane_efficiency(d, width)),
            "sorted_by_count": stats(warp_D(ds, width), lane_efficiency(ds, width)),
            "hist_bins": "%d equal bins of [0, 1]" % bins}
