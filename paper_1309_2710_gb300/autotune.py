"""Autotuner for the launch shape of the integrator.

For one mechanism, method and precision it times kin_integrate on a sample
of the caller's cells over the candidate shapes:
  block_threads  32 .. 128 lanes per block (one cell per lane),
  blocks_per_sm  persistent blocks per SM (only shapes that fit),
  staging        per-lane rate scratch in the workspace or in shared memory,
  layout         one lane or one warp per cell (RKC; the warp layout chooses
                 block_threads, blocks_per_sm and the register budget),
and keeps the fastest. Results are cached per GPU and mechanism shape in a
JSON file next to the built library.
"""
from __future__ import annotations

import json
import os
from typing import Dict, Optional

import torch

from . import build as _build
from . import kin

CACHE = os.path.join(_build.OUT_DIR, "autotune.json")


def _key(mech: kin.Mechanism, method: int, precision: int, desc) -> str:
    dev = torch.cuda.get_device_name()
    n_m = int(len(desc.eff)) if hasattr(desc, "eff") else -1
    return "%s|%d|%d|%d|%d|%d" % (dev, mech.n_species, mech.n_reactions, n_m, method, precision)


def lane_candidates(full: bool = False):
    for occupancy in (kin.OCC_DEFAULT, kin.OCC_HIGH):
        for staging in (kin.STAGE_GLOBAL, kin.STAGE_SHARED, kin.STAGE_SHARED_ALL):
            for threads in ((128, 64, 32) if full else (128, 32)):
                for lanes in ((256, 384, 512, 640, 768) if full else (384, 512, 768)):
                    bps = lanes // threads
                    yield dict(block_threads=threads, blocks_per_sm=bps, staging=staging,
                               occupancy=occupancy, layout=kin.LAYOUT_LANE)


def warp_candidates(full: bool = False, method: int = kin.RKC):
    # the register budget is a choice of the RKC warp kernels only
    for occupancy in ((kin.OCC_DEFAULT, kin.OCC_HIGH) if method == kin.RKC else (kin.OCC_DEFAULT,)):
        for threads in ((64, 128, 256) if full else (128, 256)):
            for warps in ((8, 12, 16, 24, 32, 40) if full else (8, 16, 24, 32, 40)):
                bps = warps * 32 // threads
                if bps >= 1:
                    yield dict(block_threads=threads, blocks_per_sm=bps, staging=kin.STAGE_GLOBAL,
                               occupancy=occupancy, layout=kin.LAYOUT_WARP)


def candidates(full: bool = False, method: int = kin.RKC, n_reactions: int = 0):
    """Launch shapes to try; `full` adds more block sizes and lane counts.
    Mechanisms above the warp-layout threshold try warp shapes only (one lane
    per cell is an order of magnitude slower there); smaller mechanisms try
    both layouts (one warp per cell wins on calls with few cells)."""
    if n_reactions > kin.WARP_MIN_REACTIONS:
        yield from warp_candidates(full, method)
        return
    yield from lane_candidates(full)
    yield from warp_candidates(False, method)


def time_config(mech, T0, p, Y0, dt, rtol, atol, method, precision, cfg, reps=2,
                sigma=kin.SIGMA_GERSHGORIN, energy=0) -> Optional[float]:
    """Mean kernel milliseconds of kin_integrate with `cfg`, or None if the
    shape is not supported."""
    cells = int(T0.numel())
    try:
        ws = mech.workspace(method, precision, cells, cfg["block_threads"], cfg["blocks_per_sm"],
                            T0.device, cfg["staging"], cfg["occupancy"], sigma, cfg["layout"], energy)
    except kin.KinError:
        return None
    Y = torch.empty_like(Y0)
    T = torch.empty_like(T0)  # the energy equation writes T back
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    best = None
    for r in range(reps + 1):
        Y.copy_(Y0)
        T.copy_(T0)
        ev[0].record()
        try:
            kin.integrate(mech, T, p, Y, dt, rtol, atol, method, precision, workspace=ws,
                          sigma=sigma, energy=energy, **cfg)
        except kin.KinError:
            return None
        ev[1].record()
        torch.cuda.synchronize()
        ms = ev[0].elapsed_time(ev[1])
        if r > 0:
            best = ms if best is None else min(best, ms)
    return best


def tune(mech: kin.Mechanism, desc, T, p, Y, dt, rtol, atol, method, precision,
         use_cache: bool = True, verbose: bool = False, full: bool = False, reps: int = 1,
         sigma: int = kin.SIGMA_GERSHGORIN, energy: int = 0) -> Dict:
    """Best launch shape for this mechanism on the current GPU, timed on the
    given (device) cells: pass the cells of a representative call, since the
    persistent grid's tail depends on the cell count."""
    key = _key(mech, method, precision, desc) + "|%d|%d|%d|v5" % (int(T.numel()), sigma, energy)
    cache = {}
    if use_cache and os.path.exists(CACHE):
        with open(CACHE) as f:
            cache = json.load(f)
        if key in cache:
            return cache[key]
    results = []
    for cfg in candidates(full, method, mech.n_reactions):
        ms = time_config(mech, T, p, Y, dt, rtol, atol, method, precision, cfg, reps, sigma, energy)
        if verbose:
            print("autotune", cfg, ms)
        if ms is not None:
            results.append((ms, cfg))
    results.sort(key=lambda x: x[0])
    best = dict(results[0][1], ms=results[0][0], cells=int(T.numel()))
    cache[key] = best
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    with open(CACHE, "w") as f:
        json.dump(cache, f, indent=1)
    return best
