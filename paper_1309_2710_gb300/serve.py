"""Continuous-batching server for kinetics integration requests.

A request is one CFD subdomain: its cells' (T, p, Y), the flow step dt and
the tolerances, for one of the registered mechanisms. The server

* admits arrived requests in FIFO order while their device state fits a
  memory budget, and keeps that state resident until the result is back; the
  budget also holds the slots' workspaces, sized once per run for the
  largest launch a slot can make;
* groups admitted requests by mechanism/method/precision and launches each
  group's waiting requests as ONE persistent kin_integrate_batch launch on one
  of the group's stream slots as soon as a slot is free, so requests that
  arrive while others run start on another slot and overlap on the device;
* returns each request's Y and status, and records arrival, launch and
  completion times (latency = completion - arrival).

`one_launch_per_request` is the plain alternative: one kin_integrate per
request, in arrival order, on one stream, with the same kernels and launch
shape as the server's slots.

Every cell is integrated independently by the same per-lane arithmetic, so a
request's result does not depend on what it is batched with (the tests check
bitwise identity against a standalone run).
"""
from __future__ import annotations

import argparse
import json
import math
import time
from dataclasses import dataclass, field
from typing import Dict, List, Optional

import numpy as np
import torch

from . import kin, synth


@dataclass
class Request:
    rid: int
    group: str
    T: torch.Tensor  # pinned host [cells]
    p: torch.Tensor  # pinned host [cells]
    Y: torch.Tensor  # pinned host [n_species, cells], unit column stride
    dt: float
    rtol: float = 1e-6
    atol: float = 1e-10
    arrival: float = 0.0
    Y_out: Optional[torch.Tensor] = None
    status: Optional[torch.Tensor] = None
    t_admit: float = math.nan
    t_launch: float = math.nan
    t_done: float = math.nan
    _dev: Optional[tuple] = None
    _bytes: int = 0

    @property
    def cells(self) -> int:
        return int(self.T.numel())

    @property
    def latency(self) -> float:
        return self.t_done - self.arrival


@dataclass
class Group:
    """One mechanism/method/precision served together. `shape` is the launch
    shape of one slot's persistent launch (kin_opts fields block_threads,
    blocks_per_sm, staging, occupancy, layout, and the f evaluation feval): a
    slot that leaves SM resources free lets the other slots' launches run
    beside it."""
    mech: kin.Mechanism
    method: int
    precision: int
    shape: Dict[str, int] = field(default_factory=dict)
    sigma: int = kin.SIGMA_GERSHGORIN
    max_batch_cells: Optional[int] = None  # cap on one launch's cells (None: the server's)


@dataclass
class _Slot:
    stream: torch.cuda.Stream
    workspace: Optional[torch.Tensor] = None
    batch: List[Request] = field(default_factory=list)
    event: Optional[torch.cuda.Event] = None


def _h2d(dst: torch.Tensor, src: torch.Tensor):
    """Asynchronous host-to-device copy; strided 2-D sources row by row."""
    if src.dim() == 2 and not src.is_contiguous():
        for i in range(src.shape[0]):
            dst[i].copy_(src[i], non_blocking=True)
    else:
        dst.copy_(src, non_blocking=True)


class Server:
    def __init__(self, groups: Dict[str, Group], budget_bytes: int, slots_per_group: int = 2,
                 max_instances: int = kin.MAX_INSTANCES, max_batch_cells: int = 1 << 21,
                 device=None):
        self.groups = groups
        self.budget = int(budget_bytes)
        self.max_instances = min(max_instances, kin.MAX_INSTANCES)
        self.max_batch_cells = max_batch_cells
        self.device = device or torch.device("cuda")
        self.slots = {g: [_Slot(torch.cuda.Stream(device=self.device)) for _ in range(slots_per_group)]
                      for g in groups}
        self.used = 0        # device bytes of admitted requests' state
        self.peak_used = 0   # the largest `used` seen
        self.ws_bytes = 0    # device bytes of the slots' workspaces

    def _cap(self, gname: str) -> int:
        return self.groups[gname].max_batch_cells or self.max_batch_cells

    def _size_workspaces(self, requests: List[Request]):
        """Allocate every slot's workspace once, for the largest launch it can
        make in this run: the group's per-launch cell cap (or all of the
        group's cells, if fewer), or a single larger request."""
        self.ws_bytes = 0
        for gname, slots in self.slots.items():
            g = self.groups[gname]
            sizes = [r.cells for r in requests if r.group == gname]
            cells = max(max(sizes, default=0), min(self._cap(gname), sum(sizes)))
            sh = g.shape
            need = g.mech.workspace_bytes(g.method, g.precision, cells, sh.get("block_threads", 0),
                                          sh.get("blocks_per_sm", 0), sh.get("staging", 0),
                                          sh.get("occupancy", 0), g.sigma, sh.get("layout", 0))
            for slot in slots:
                if slot.workspace is None or slot.workspace.numel() < need:
                    slot.workspace = torch.empty(need, dtype=torch.uint8, device=self.device)
                self.ws_bytes += slot.workspace.numel()

    def request_bytes(self, r: Request) -> int:
        nS = self.groups[r.group].mech.n_species
        return r.cells * ((nS + 2) * 8 + 1)

    # -------------------------------------------------------------- steps --
    def _admit(self, r: Request, now: float):
        n, nS = r.cells, self.groups[r.group].mech.n_species
        d = self.device
        r._dev = (torch.empty(n, dtype=torch.float64, device=d),
                  torch.empty(n, dtype=torch.float64, device=d),
                  torch.empty((nS, n), dtype=torch.float64, device=d),
                  torch.empty(n, dtype=torch.uint8, device=d))
        r.Y_out = torch.empty((nS, n), dtype=torch.float64, pin_memory=True)
        r.status = torch.empty(n, dtype=torch.uint8, pin_memory=True)
        r._bytes = self.request_bytes(r)
        self.used += r._bytes
        self.peak_used = max(self.peak_used, self.used)
        r.t_admit = now

    def _launch(self, gname: str, slot: _Slot, batch: List[Request], now: float):
        g = self.groups[gname]
        with torch.cuda.stream(slot.stream):
            parts = []
            for r in batch:
                Td, pd, Yd, sd = r._dev
                _h2d(Td, r.T)
                _h2d(pd, r.p)
                _h2d(Yd, r.Y)
                parts.append(kin.Cells(Td, pd, Yd, r.dt, r.rtol, r.atol, sd))
                r.t_launch = now
            kin.integrate_batch(g.mech, parts, g.method, g.precision, workspace=slot.workspace,
                                stream=slot.stream, sigma=g.sigma, **g.shape)
            for r in batch:
                r.Y_out.copy_(r._dev[2], non_blocking=True)
                r.status.copy_(r._dev[3], non_blocking=True)
            slot.event = torch.cuda.Event()
            slot.event.record(slot.stream)
        slot.batch = batch

    def _complete(self, slot: _Slot, now: float):
        for r in slot.batch:
            r.t_done = now
            r._dev = None
            self.used -= r._bytes
        slot.batch = []
        slot.event = None

    # ---------------------------------------------------------------- run --
    def run(self, requests: List[Request]) -> List[Request]:
        """Serve `requests` (arrival times in seconds from the start of the
        call, in wall-clock time). Returns them with results and times."""
        todo = sorted(requests, key=lambda r: r.arrival)
        self._size_workspaces(todo)
        for r in todo:
            if self.ws_bytes + self.request_bytes(r) > self.budget:
                raise ValueError("request %d needs more memory than the budget" % r.rid)
        waiting: List[Request] = []  # arrived, not admitted (FIFO)
        ready: Dict[str, List[Request]] = {g: [] for g in self.groups}
        nxt, done = 0, 0
        t0 = time.perf_counter()
        while done < len(todo):
            now = time.perf_counter() - t0
            while nxt < len(todo) and todo[nxt].arrival <= now:
                waiting.append(todo[nxt])
                nxt += 1
            while waiting and self.ws_bytes + self.used + self.request_bytes(waiting[0]) <= self.budget:
                r = waiting.pop(0)
                self._admit(r, now)
                ready[r.group].append(r)
            progressed = False
            for gname, slots in self.slots.items():
                for slot in slots:
                    if slot.event is not None and slot.event.query():
                        done += len(slot.batch)
                        self._complete(slot, now)
                        progressed = True
                    if slot.event is None and ready[gname]:
                        batch, cells = [], 0
                        q = ready[gname]
                        cap = self._cap(gname)
                        while q and len(batch) < self.max_instances and (
                                not batch or cells + q[0].cells <= cap):
                            r = q.pop(0)
                            batch.append(r)
                            cells += r.cells
                        self._launch(gname, slot, batch, now)
                        progressed = True
            if not progressed:
                time.sleep(20e-6)
        return todo


def one_launch_per_request(groups: Dict[str, Group], requests: List[Request], device=None):
    """Plain FIFO: one kin_integrate per request on one stream, each waited for."""
    device = device or torch.device("cuda")
    stream = torch.cuda.Stream(device=device)
    todo = sorted(requests, key=lambda r: r.arrival)
    ws: Dict[str, torch.Tensor] = {}
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for r in todo:
            while time.perf_counter() - t0 < r.arrival:
                time.sleep(20e-6)
            g = groups[r.group]
            n, nS = r.cells, g.mech.n_species
            r.t_launch = time.perf_counter() - t0
            Td = torch.empty(n, dtype=torch.float64, device=device)
            pd = torch.empty(n, dtype=torch.float64, device=device)
            Yd = torch.empty((nS, n), dtype=torch.float64, device=device)
            sd = torch.empty(n, dtype=torch.uint8, device=device)
            _h2d(Td, r.T)
            _h2d(pd, r.p)
            _h2d(Yd, r.Y)
            sh = g.shape
            need = g.mech.workspace_bytes(g.method, g.precision, n, sh.get("block_threads", 0),
                                          sh.get("blocks_per_sm", 0), sh.get("staging", 0),
                                          sh.get("occupancy", 0), g.sigma, sh.get("layout", 0))
            if r.group not in ws or ws[r.group].numel() < need:
                ws[r.group] = torch.empty(need, dtype=torch.uint8, device=device)
            kin.integrate(g.mech, Td, pd, Yd, r.dt, r.rtol, r.atol, g.method, g.precision,
                          status=sd, workspace=ws[r.group], stream=stream, sigma=g.sigma, **sh)
            r.Y_out = torch.empty((nS, n), dtype=torch.float64, pin_memory=True)
            r.status = torch.empty(n, dtype=torch.uint8, pin_memory=True)
            r.Y_out.copy_(Yd, non_blocking=True)
            r.status.copy_(sd, non_blocking=True)
            stream.synchronize()
            r.t_done = time.perf_counter() - t0
    return todo


# ------------------------------------------------------- serving workload --
class StatePool:
    """Pinned, species-major pool of seeded initial states per mechanism;
    a request of n cells views n consecutive pool cells."""

    def __init__(self, name: str, mech, cells: int, seed_offset: int = 500):
        T, p, Y = synth.workload_states(name, mech, cells=cells, seed_offset=seed_offset)
        self.T = torch.as_tensor(T).pin_memory()
        self.p = torch.as_tensor(p).pin_memory()
        self.Y = torch.as_tensor(Y).contiguous().pin_memory()
        self.cells = cells

    def view(self, off: int, n: int):
        return self.T[off:off + n], self.p[off:off + n], self.Y[:, off:off + n]


def make_requests(n: int, pools: Dict[str, StatePool], seed: int = 3005, loads_rate=None):
    """The serving workload (Section 3 setup recast as requests): mechanism
    13- or 53-species (p = 0.5), cells log-uniform in [1024, 65536], dt
    log-uniform in [1e-7, 1e-5] s, rtol 1e-6. Arrival times are 0 unless a
    Poisson rate (requests/s) is given."""
    spec = synth.serve_requests(n, seed=seed)
    rng = np.random.default_rng(seed + 1)
    t = 0.0
    out = []
    for i, (g, cells, dt) in enumerate(spec):
        pool = pools[g]
        off = int(rng.integers(0, pool.cells - cells + 1))
        T, p, Y = pool.view(off, cells)
        if loads_rate:
            t += rng.exponential(1.0 / loads_rate)
        out.append(Request(i, g, T, p, Y, dt, arrival=t))
    return out


def percentiles(reqs: List[Request]):
    lat = np.array([r.latency for r in reqs])
    cells = sum(r.cells for r in reqs)
    span = max(r.t_done for r in reqs) - min(r.arrival for r in reqs)
    return {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "throughput_cells_per_s": cells / span, "requests": len(reqs), "cells": int(cells)}


# Per-slot launch shapes of the serving groups: about a third of an SM's
# registers each, so that launches of the other slots and group fit beside.
# Each launch is capped (about 75 ms of work at the 13-species and 190 ms at
# the 53-species throughput), so a request that arrives behind a large batch
# waits for a short launch rather than a long one.
SERVE_BATCH_CELLS = {"h2co_13sp_rkc": 131072, "ch4_53sp_rkc_mixed": 32768}
SERVE_SLOTS = 4
# The f evaluation is pinned per group (the automatic choice depends on the
# launch's cell count, and a request must get the same bits in any batch).
SERVE_SHAPES = {
    "h2co_13sp_rkc": dict(block_threads=128, blocks_per_sm=2, occupancy=kin.OCC_HIGH,
                          layout=kin.LAYOUT_LANE, feval=kin.FEVAL_GENERATED),
    "ch4_53sp_rkc_mixed": dict(block_threads=256, blocks_per_sm=1, layout=kin.LAYOUT_WARP,
                               feval=kin.FEVAL_TABLE),
}


def default_groups():
    groups, pools = {}, {}
    for name in ("h2co_13sp_rkc", "ch4_53sp_rkc_mixed"):
        w = synth.WORKLOADS[name]
        m = synth.workload_mechanism(name)
        groups[name] = Group(kin.Mechanism(m), w["method"], w["precision"], dict(SERVE_SHAPES[name]),
                             w["sigma"], SERVE_BATCH_CELLS[name])
        pools[name] = StatePool(name, m, 65536 + 1024)
    return groups, pools


def benchmark(requests: int = 2000, loads=(0.5, 0.8, 0.95), budget_gb: float = 16.0,
              slots: int = SERVE_SLOTS, saturation_requests: Optional[int] = None):
    """The serving measurement: the saturated throughput of continuous
    batching (every request arrives at t = 0; `saturation_requests` of them,
    default `requests`), then at each offered load (a fraction of that
    throughput, Poisson arrivals) `requests` requests served by continuous
    batching and by one launch per request, with p50/p99 latency and
    throughput of each."""
    groups, pools = default_groups()
    budget = int(budget_gb * (1 << 30))
    # warm up both paths (module loads, workspaces, pinned pools)
    warm = make_requests(8, pools, seed=7)
    Server(groups, budget, slots).run(warm)
    one_launch_per_request(groups, make_requests(4, pools, seed=8))
    torch.cuda.synchronize()
    sat_reqs = make_requests(saturation_requests or requests, pools)
    srv = Server(groups, budget, slots)
    sat = percentiles(srv.run(sat_reqs))
    mean_cells = np.mean([r.cells for r in make_requests(requests, pools)])
    out = {"saturated": sat, "budget_bytes": budget, "workspace_bytes": srv.ws_bytes,
           "peak_state_bytes": srv.peak_used, "slots_per_group": slots,
           "batch_cells_cap": dict(SERVE_BATCH_CELLS), "loads": []}
    for load in loads:
        rate = load * sat["throughput_cells_per_s"] / mean_cells
        a = percentiles(Server(groups, budget, slots).run(make_requests(requests, pools, loads_rate=rate)))
        b = percentiles(one_launch_per_request(groups, make_requests(requests, pools, loads_rate=rate)))
        out["loads"].append({"load": load, "offered_requests_per_s": rate,
                             "continuous_batching": a, "one_launch_per_request": b})
    for g in groups.values():
        g.mech.close()
    return out


def main():
    ap = argparse.ArgumentParser(description="continuous-batching serving benchmark")
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--loads", default="0.5,0.8,0.95")
    ap.add_argument("--budget-gb", type=float, default=16.0)
    ap.add_argument("--slots", type=int, default=SERVE_SLOTS)
    args = ap.parse_args()
    from . import build as _b
    _b.build()
    out = benchmark(args.requests, [float(x) for x in args.loads.split(",") if x], args.budget_gb,
                    args.slots)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
