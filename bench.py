"""Benchmark: cell-ODEs integrated over one flow step per second on GB300.

Default workload: the 13-species / 54-reaction synthetic mechanism, RKC with
a Gershgorin spectral radius, 262144 cells, dt = 1e-6 s, rtol 1e-6,
atol 1e-10, FP64. One step = one kin_integrate call over every cell (the
whole hot path: source terms, RKC stages, spectral radius, error control),
starting from the same initial state every step (the integrator restarts per
flow step).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl kin|reference]

Prints one JSON line. With --impl reference the plain FP64 CPU oracle is
timed on the host cores instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1309_2710_gb300 import synth  # noqa: E402

METRIC = "cell-ODEs integrated over Δt per sec per GB300 at rtol 1e-6"
UNIT = "cell-ODEs/s"
L2_FLUSH_BYTES = 256 << 20

# The FP64 pipe binds this path (the FP32 pipe can bind the mixed path's
# rate arithmetic; the pipe with the larger operations / peak binds). The
# peaks are measured in every run by the dependent-FMA probe of
# include/kin_peaks.h on the GPU being timed (measure_peaks). Only if that
# probe fails do the nominal figures below stand in, and the line says so:
# 2 FP64 and 128 FP32 FMA lanes per SM per clock x 152 SMs x 2070 MHz.
FP64_LANES_PER_SM = 2
FP32_LANES_PER_SM = 128
SM_COUNT = 152
SM_MAX_MHZ = 2070.0

# DRAM bytes (read + write) per launch of the dominant kernel from one ncu
# capture (profiles/), valid only for the kernel sources whose hash is the key
# and for the captured launch shape (block threads, blocks per SM, staging,
# register budget, layout) and f evaluation: (workload, shape, f) -> (bytes,
# cells in the captured launch). A capture on fewer cells than the benchmarked
# workload is scaled by the cell count.
TRAFFIC = {
    "d4328964f870": {
        ("h2co_13sp_rkc", (32, 16, 0, 0, 1), "generated"): (7332879872 + 13668991488, 262144),
        ("ch4_53sp_rkc_mixed", (256, 5, 0, 1, 2), "tables"): (348273920 + 1347731968, 65536),
    },
}


def traffic_for(name, shape_key, fname, cells):
    """DRAM bytes per launch for this workload and launch shape: the capture of
    the same shape, else of the same kernel variant (staging, register budget,
    layout) with the same resident lanes per SM; scaled to `cells`. Returns
    (bytes or None, captured shape or None)."""
    tab = TRAFFIC.get(kernel_hash(), {})
    hit = tab.get((name, shape_key, fname))
    cap = shape_key
    if hit is None:
        for (nm, sk, fn), v in tab.items():
            if (nm == name and fn == fname and sk[2:] == shape_key[2:]
                    and sk[0] * sk[1] == shape_key[0] * shape_key[1]):
                hit, cap = v, sk
                break
    if hit is None:
        return None, None
    return hit[0] * cells / hit[1], list(cap)


# sources that define no integrator kernel: the host side of the ABI
# (argument checks, launch choices) and the arithmetic-peak probe
HOST_ONLY = ("abi.cu", "no_alloc.cu", "peaks.cu")


def kernel_hash() -> str:
    """Hash of the sources that define kernel code (device templates, their
    instantiations, the generator of the run-time compiled f, and the layout
    of the warp f's gather tables)."""
    d = os.path.join(ROOT, "paper_1309_2710_gb300", "csrc")
    h = hashlib.sha1()
    for f in sorted(os.listdir(d)):
        if (f.endswith((".cu", ".cuh")) or f == "seg_tables.h") and f not in HOST_ONLY:
            h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:12]


# ------------------------------------------------------ algorithmic work ---
def feval_ops(m) -> int:
    """FP64 operations of one evaluation of f in its minimal fused form
    (an FMA, add, multiply or divide is one operation)."""
    nS = m.n_species
    o = 3 * nS + 1  # Y/W, sum, rho, C
    for j in range(m.n_reactions):
        o += int(np.count_nonzero(m.reac[j] >= 0))
        if m.rtype[j] == synth.THIRD_BODY:
            o += nS + 1  # [M] as nS fused multiply-adds, times [M]
        elif m.rtype[j] == synth.FALLOFF:
            o += nS + 4  # [M], Pr, 1 + Pr, Pr/(1+Pr), times
    for i in range(nS):
        for j in range(m.n_reactions):
            if int(np.sum(m.prod[j] == i)) != int(np.sum(m.reac[j] == i)):
                o += 1  # one fused multiply-add per net nonzero
    o += nS + 1  # 1/rho, dY_i/dt = (W_i omega_i) / rho (W_i folded into the coefficients)
    return o


def feval_ops_energy(m) -> int:
    """feval_ops plus the work the energy equation adds to one evaluation: the
    rate constants from T (2 per reaction for the exponent, one exp; falloff
    reactions a second exponent and exp), log T and the reciprocals (3), the
    enthalpy sum and mixture heat capacity (3 per species) and dT/dt (3). An
    exp or log counts as one operation, so this is a lower bound."""
    n_fo = int(np.count_nonzero(m.rtype == synth.FALLOFF))
    return feval_ops(m) + 3 * m.n_reactions + 3 * n_fo + 3 + 3 * m.n_species + 3


def algorithmic_work(m, method, precision, sigma, stats, energy=False):
    """Algorithmic operations of one call, from the per-cell counts (f
    evaluations, accepted and rejected steps, spectral-radius estimates), as
    (FP64 lane-ops, FP32 lane-ops, exact). An FMA, add, multiply or divide is
    one operation; conversions are not counted.

    f costs feval_ops(m). In the mixed path its rate arithmetic is FP32 and
    only the final scaling dY/dt = W omega / rho (nS + 1) is FP64, while
    every spectral-radius evaluation is FP64, including the re-evaluation of
    f(y) that each estimate starts from. RKC vector work (FP64): per attempt
    w_1 and the error estimate and norm (8 nS), per further stage the
    recursion (5 nS); Gershgorin: 3 nS per column; power method: 4 nS per
    product; initial step 6 nS. The per-cell counters split the f evaluations
    between spectral-radius estimates and rate evaluations, so the count is
    exact (with the energy equation an exp or log counts as one operation)."""
    nS = m.n_species + (1 if energy else 0)  # state length
    fo = feval_ops_energy(m) if energy else feval_ops(m)
    mixed = precision == synth.MIXED
    # FP64 part of one rate-type f evaluation: in the mixed path the final
    # scaling (and with the energy equation the exponents and the enthalpy
    # sums) stay FP64
    f64 = (m.n_species + 1 + (fo - feval_ops(m) if energy else 0)) if mixed else fo
    f32 = fo - f64
    nfe = stats[:, 0].astype(np.float64)
    att = (stats[:, 1] + stats[:, 2]).astype(np.float64)
    nsig = stats[:, 3].astype(np.float64)
    if method != synth.RKC:
        return float((nfe * f64 + att * 38 * nS).sum()), float((nfe * f32).sum()), True
    base = 1 if mixed else 0
    # the fifth statistic counts the f evaluations inside the spectral-radius
    # estimates (Gershgorin columns or power products, plus the FP64 base
    # evaluation of the mixed path), so the split is exact
    sig_evals = stats[:, 4].astype(np.float64)
    per_eval = 3 * nS if sigma == synth.GERSHGORIN else 4 * nS
    sig_vec = (sig_evals - nsig * base) * per_eval
    exact = not energy  # an exp or log of the energy path counts as one operation
    rate_evals = nfe - sig_evals            # f(y0), the initial-step probe, the stages
    stages = rate_evals - 2
    vec = (stages - att) * 5 * nS + att * 8 * nS + sig_vec + 6 * nS
    ops64 = (rate_evals * f64 + sig_evals * fo + vec).sum()
    ops32 = (rate_evals * f32).sum()
    return float(ops64), float(ops32), exact


def contract_flops(m, method, precision, stats, energy=False):
    """Algorithmic flops of one call in the hot-path contract's count (an FMA
    is 2 flops), from the per-cell counters. Per f evaluation
    F = 4 nS + 2 nR + 2 nS nM + 6 nFO + 8 nR + 2 nS (mixture and
    concentrations, rates of progress, third-body sums over the nM
    third-body and falloff reactions, falloff blending, the stoichiometric
    gather, dY/dt); RKC adds 10 nS per stage, 14 nS per attempt and 2 nS^2
    per spectral-radius estimate, RKCK 60 nS per attempt. Returns (FP64
    flops, FP32 flops): in the mixed path a rate evaluation is FP32 but for
    its final 2 nS, and every spectral-radius evaluation is FP64. With the
    energy equation nS counts T too and the per-evaluation rate constants
    are not counted (a lower bound)."""
    nS = m.n_species + (1 if energy else 0)
    nR = m.n_reactions
    n_m = int(np.count_nonzero(m.rtype != synth.PLAIN))
    n_fo = int(np.count_nonzero(m.rtype == synth.FALLOFF))
    F = 4 * nS + 2 * nR + 2 * nS * n_m + 6 * n_fo + 8 * nR + 2 * nS
    nfe = stats[:, 0].astype(np.float64)
    att = (stats[:, 1] + stats[:, 2]).astype(np.float64)
    nsig = stats[:, 3].astype(np.float64)
    sig_evals = stats[:, 4].astype(np.float64)
    mixed = precision == synth.MIXED
    if method != synth.RKC:
        rate = nfe * F
        vec = att * 60 * nS
    else:
        rate = (nfe - sig_evals) * F
        stages = nfe - sig_evals - 2  # f(y0) and the initial-step probe are not stages
        vec = stages * 10 * nS + att * 14 * nS + nsig * 2 * nS * nS + sig_evals * F
    f32 = (rate - (nfe - sig_evals if method == synth.RKC else nfe) * 2 * nS) if mixed else 0.0 * rate
    f64 = rate + vec - f32
    return float(f64.sum()), float(f32.sum())


def measure_peaks(gpu_index, stream=None):
    """FP64 and FP32 FMA rates of this GPU from the dependent-FMA probe
    (include/kin_peaks.h), each the best of three ~0.3 s runs, with the SM
    clock sampled while it runs. Returns a dict (rates in FMA/s), or None if
    the probe is not available."""
    try:
        from paper_1309_2710_gb300 import peaks
        with ClockSampler(gpu_index) as clk:
            peaks.fma_rate(peaks.FP64, 20000)
            r64 = max(peaks.fma_rate(peaks.FP64, 150000)[1] for _ in range(3))
            r32 = max(peaks.fma_rate(peaks.FP32, 10000000)[1] for _ in range(3))
        return {"fp64_fma_per_s": r64, "fp32_fma_per_s": r32, "clocks": clk.summary()}
    except Exception as e:  # noqa: BLE001 - the line then says the peaks are nominal
        print("peak probe failed: %s" % e, file=sys.stderr)
        return None


def accuracy(m, Yg, Yo, stg, sto, stag, stao, atol, rtol, Tg=None, To=None):
    """Errors of the GPU result against the FP64 oracle on the same cells:
    per species the maximum of |dY| / max(|Y_ref|, atol) (the hot-path
    contract's metric) and of |dY| / max(|Y_ref|, atol/rtol) (the
    integrator's own weighting), over all cells and over the cells whose
    decision trace equals the oracle's."""
    e_a = np.abs(Yg - Yo) / np.maximum(np.abs(Yo), atol)
    e_t = np.abs(Yg - Yo) / np.maximum(np.abs(Yo), atol / rtol)
    same = (stag == stao).all(axis=1)
    # accepted and rejected step counts equal to the oracle's (the FP32 rates
    # of the mixed path move the f-evaluation counts of every cell, so its
    # decision identity is read from the steps)
    steps = (stag[:, 1:3] == stao[:, 1:3]).all(axis=1)
    et = e_t.max(axis=0)
    out = {"cells": int(Yo.shape[1]), "trace_divergent_cells": int((~same).sum()),
           "step_count_divergent_cells": int((~steps).sum()),
           "max_err_tol_weighted_steps_equal": float(et[steps].max()) if steps.any() else None,
           "max_err_tol_weighted_steps_differ": float(et[~steps].max()) if (~steps).any() else None,
           "cells_over_1e-5_tol_weighted": int((et > 1e-5).sum()),
           "status_equal": bool(np.array_equal(stg, sto)),
           "max_err": float(e_a.max()), "max_err_tol_weighted": float(e_t.max()),
           "max_err_trace_identical": float(e_a[:, same].max()) if same.any() else None,
           "per_species_max_err": [float(x) for x in e_a.max(axis=1)],
           "per_species_max_err_tol_weighted": [float(x) for x in e_t.max(axis=1)],
           "species": list(m.names),
           "metric": "|Y_gpu - Y_oracle| / max(|Y_oracle|, atol); tol_weighted: / max(|Y_oracle|, atol/rtol)"}
    if Tg is not None:
        out["T_max_rel_err"] = float((np.abs(Tg - To) / To).max())
    return out


# ------------------------------------------------------------- clocks ---
class ClockSampler:
    """nvidia-smi clocks and throttle reasons every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        mhz, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                mhz.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not mhz:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(mhz), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(mhz)}


# ---------------------------------------------------------- CPU oracle ---
def oracle_method(w):
    """The oracle's method code for a workload (2 = RKC with power sigma)."""
    if w["method"] == synth.RKCK:
        return 0
    return 2 if w["sigma"] == synth.POWER else 1


def oracle_rate(name, cells_target_s=10.0, max_cells=None, seed_offset=0, nthreads=0, result=None,
                cells=None, order="random"):
    """Time the FP64 oracle on the host cores (all of them, or `nthreads`) on
    a bounded sample of the workload: the first n cells of the same states.
    Returns (cells/s, threads, sample description); with a `result` dict,
    stores the sample's n and the oracle's outputs there (Y, status, stats
    and, with the energy equation, T)."""
    import oracle
    w = synth.WORKLOADS[name]
    m = synth.workload_mechanism(name)
    om = oracle.Mech(m)
    total = cells or w["cells"]
    T, p, Y = synth.workload_states(name, m, cells=total, seed_offset=seed_offset,
                                    sort_by_T=order == "sorted")
    probe = min(2048 if nthreads == 0 else 64, total)
    t0 = time.perf_counter()
    meth = oracle_method(w)
    en = bool(w.get("energy"))
    nt = oracle.integrate(om, T[:probe], p[:probe], Y[:, :probe], w["dt"], w["rtol"],
                          w["atol"], meth, nthreads=nthreads, energy=en)[3]
    per_cell = (time.perf_counter() - t0) / probe
    n = int(min(total if max_cells is None else max_cells, max(probe, cells_target_s / per_cell)))
    t0 = time.perf_counter()
    r = oracle.integrate(om, T[:n], p[:n], Y[:, :n], w["dt"], w["rtol"], w["atol"], meth,
                         nthreads=nthreads, energy=en)
    el = time.perf_counter() - t0
    nt = r[3]
    if result is not None:
        result.update(n=n, Y=r[0], status=r[1], stats=r[2], T=r[4] if en else None)
    return n / el, nt, "first %d of the %d cells of %s (same seeds), %.1f s wall" % (n, total, name, el)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    name = args.workload
    w = synth.WORKLOADS[name]
    m = synth.workload_mechanism(name)
    om = oracle.Mech(m)
    T, p, Y = synth.workload_states(name, m)
    # bounded per-step sample sized from a probe so K+W steps take ~2 min
    probe = 1024
    t0 = time.perf_counter()
    meth = oracle_method(w)
    en = bool(w.get("energy"))
    oracle.integrate(om, T[:probe], p[:probe], Y[:, :probe], w["dt"], w["rtol"], w["atol"], meth,
                     energy=en)
    per_cell = (time.perf_counter() - t0) / probe
    budget = 120.0 / max(1, args.steps + args.warmup)
    n = int(min(w["cells"], max(probe, budget / per_cell)))
    for _ in range(args.warmup):
        oracle.integrate(om, T[:n], p[:n], Y[:, :n], w["dt"], w["rtol"], w["atol"], meth, energy=en)
    times = []
    nt = 1
    for _ in range(args.steps):
        t0 = time.perf_counter()
        nt = oracle.integrate(om, T[:n], p[:n], Y[:, :n], w["dt"], w["rtol"], w["atol"], meth,
                              energy=en)[3]
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = n * len(times) / tot
    sample = "first %d of the %d cells per step" % (n, w["cells"])
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(name, n),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": nt, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def workload_config(name, cells, sigma=None, order="random"):
    w = synth.WORKLOADS[name]
    sigma = w["sigma"] if sigma is None else sigma
    rkc = "RKC (%s sigma)" % ("power-method" if sigma == synth.POWER else "Gershgorin FD")
    return {"workload": "%s: %d species / %d reactions, %s %s%s, %d cells, dt %g s, rtol %g, atol %g"
                        % (name, w["n_species"], w["n_reactions"],
                           rkc if w["method"] == synth.RKC else "RKCK",
                           "FP64" if w["precision"] == synth.FP64 else "mixed FP32/FP64",
                           ", constant-pressure energy equation" if w.get("energy") else "",
                           cells, w["dt"], w["rtol"], w["atol"]),
            "energy_equation": bool(w.get("energy")),
            "cells": cells, "method": "RKC" if w["method"] == synth.RKC else "RKCK",
            "precision": "fp64" if w["precision"] == synth.FP64 else "mixed",
            "l2": "flushed between steps (256 MiB write)", "cell_order": "random (as drawn)" if order == "random" else
            "similar (sorted by temperature, the paper's 'similar' initial conditions)"}


# ------------------------------------------------------------ GPU arm ---
def rank_states(name, m, cells_per_rank, world, rank, order="random"):
    """This rank's block of the whole job. The job is world x cells_per_rank
    cells of one seeded draw (so the per-GPU work stays fixed as ranks are
    added: weak scaling); the cells are independent (Section 2.1), so each
    rank takes its contiguous block (shard.shard_cells) and integrates it
    with no exchange. Returns (start, stop, T, p, Y)."""
    from paper_1309_2710_gb300 import shard
    total = world * cells_per_rank
    T, p, Y = synth.workload_states(name, m, cells=total, sort_by_T=order == "sorted")
    a, b = shard.shard_cells(total, world, rank)
    return a, b, T[a:b], p[a:b], np.ascontiguousarray(Y[:, a:b])


def roofline(m, method, prec, sigma, stats, energy, kernel_ms, pk, world=1):
    """The dominant launch against the binding arithmetic pipe, in two
    counts: the hot-path contract's flops (FMA = 2; contract_flops) against
    twice the measured FMA rate, and this build's lane operations (an FMA,
    add, multiply or divide is one; algorithmic_work) against the FMA rate.
    The FP64 and FP32 pipes run concurrently; the one with the larger work /
    peak binds."""
    ops64, ops32, exact = algorithmic_work(m, method, prec, sigma, stats, energy)
    fl64, fl32 = contract_flops(m, method, prec, stats, energy)
    if pk:
        f64, f32 = pk["fp64_fma_per_s"], pk["fp32_fma_per_s"]
        basis = ("measured: dependent-FMA probe (include/kin_peaks.h) on this GPU in this run, "
                 "median SM clock %s MHz" % pk["clocks"].get("sm_mhz"))
    else:
        f64 = FP64_LANES_PER_SM * SM_COUNT * SM_MAX_MHZ * 1e6
        f32 = FP32_LANES_PER_SM * SM_COUNT * SM_MAX_MHZ * 1e6
        basis = "nominal (the probe failed): 2 FP64 / 128 FP32 FMA lanes/SM/clk x 152 SMs x 2070 MHz"
    t = kernel_ms * 1e-3
    b64 = fl64 / f64 >= fl32 / f32
    ach = world * (fl64 if b64 else fl32) / t / 1e9
    peak = world * 2 * (f64 if b64 else f32) / 1e9
    l64 = ops64 / f64 >= ops32 / f32
    lach = world * (ops64 if l64 else ops32) / t / 1e9
    lpeak = world * (f64 if l64 else f32) / 1e9
    return {"bound": "alu", "achieved": ach, "peak": peak,
            "unit": "GFLOP/s %s (FMA = 2 flops)" % ("FP64" if b64 else "FP32"), "frac": ach / peak,
            "count": "hot-path contract: per f 4nS+2nR+2nS*nM+6nFO+8nR+2nS; RKC 10nS/stage, 14nS/attempt, "
                     "2nS^2/sigma estimate; RKCK 60nS/attempt; oracle-equal per-cell counters",
            "peak_basis": basis, "kernel_ms": kernel_ms, "fp64_flops_per_launch": fl64,
            "fp32_flops_per_launch": fl32,
            "lane_ops": {"achieved": lach, "peak": lpeak, "frac": lach / lpeak,
                         "unit": "G %s lane-ops/s (FMA, add, multiply, divide = 1)" % ("FP64" if l64 else "FP32"),
                         "fp64_ops_per_launch": ops64, "fp32_ops_per_launch": ops32,
                         "count": "exact" if exact else "lower bound"}}


def run_kin(args):
    import torch
    import torch.distributed as dist
    from paper_1309_2710_gb300 import build as kbuild
    kbuild.build()
    from paper_1309_2710_gb300 import kin

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    name = args.workload
    w = synth.WORKLOADS[name]
    m = synth.workload_mechanism(name)
    cells_per_rank = args.cells or w["cells"]
    a0, b0, T, p, Y0 = rank_states(name, m, cells_per_rank, world, rank, args.order)
    cells = b0 - a0
    km = kin.Mechanism(m)
    method, prec = w["method"], w["precision"]
    sigma = w["sigma"] if args.sigma == "default" else (synth.POWER if args.sigma == "power"
                                                         else synth.GERSHGORIN)
    energy = int(bool(w.get("energy")))
    T0d = torch.as_tensor(T, device=dev)
    Td = T0d.clone()  # integrated (and reset every step) with the energy equation
    pd = torch.as_tensor(p, device=dev)
    Y0d = torch.as_tensor(Y0, device=dev).contiguous()
    Yd = torch.empty_like(Y0d)
    st = torch.zeros(cells, dtype=torch.uint8, device=dev)
    sta = torch.zeros((cells, kin.NSTATS), dtype=torch.int32, device=dev)
    shape = dict(block_threads=0, blocks_per_sm=0, staging=kin.STAGE_GLOBAL, occupancy=kin.OCC_DEFAULT,
                 layout=kin.LAYOUT_AUTO)
    if args.shape:
        v = [int(x) for x in args.shape.split(",")]
        shape = dict(zip(("block_threads", "blocks_per_sm", "staging", "occupancy", "layout"), v))
        shape.setdefault("layout", kin.LAYOUT_AUTO)
    elif not args.no_tune:
        # launch shape from the autotuner (cached per GPU, mechanism shape and
        # cell count), timed on this workload outside the timed region
        from paper_1309_2710_gb300 import autotune
        best = autotune.tune(km, m, T0d, pd, Y0d, w["dt"], w["rtol"], w["atol"], method, prec,
                             sigma=sigma, energy=energy)
        shape = {k: best[k] for k in shape}
    if args.feval != "auto":
        shape["feval"] = kin.FEVAL_TABLE if args.feval == "table" else kin.FEVAL_GENERATED
    ws = km.workspace(method, prec, cells, shape["block_threads"], shape["blocks_per_sm"], dev,
                      shape["staging"], shape["occupancy"], sigma, shape["layout"], energy)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step(ev=None):
        flush.zero_()
        Yd.copy_(Y0d)
        if energy:
            Td.copy_(T0d)
        if ev:
            ev[0].record(stream)
        kin.integrate(km, Td, pd, Yd, w["dt"], w["rtol"], w["atol"], method, prec,
                      status=st, stats=sta, workspace=ws, stream=stream, sigma=sigma,
                      energy=energy, **shape)
        if ev:
            ev[1].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # the arithmetic peaks of this GPU, measured before the timed region
    pk = measure_peaks(local)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_start.record(stream)
        for k in range(args.steps):
            step(evs[k])
        t_end.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms_total = t_start.elapsed_time(t_end)
    kern_ms = [a.elapsed_time(b) for a, b in evs]
    tmax = torch.tensor([ms_total, float(np.mean(kern_ms))], device=dev, dtype=torch.float64)
    if world > 1:
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    ms_step = float(tmax[0].item()) / args.steps
    value = world * cells_per_rank / (ms_step * 1e-3)

    stats = sta.cpu().numpy()
    status = st.cpu().numpy()
    kavg = float(tmax[1].item())
    roof = roofline(m, method, prec, sigma, stats, energy, kavg, pk, world)
    shape_key = tuple(int(shape[k]) for k in ("block_threads", "blocks_per_sm", "staging", "occupancy",
                                                 "layout"))
    fname = feval_name(km, prec, shape, cells, layout_name(km, method, shape, cells), energy)
    tr, tr_shape = traffic_for(name, shape_key, fname, cells)
    roof.update(traffic=tr, traffic_capture_shape=tr_shape,
                kernel="kin_integrate launch (init + sort + integrate kernels, %s layout, %s f)"
                       % (layout_name(km, method, shape, cells), fname))
    Yg = Yd.cpu().numpy()
    Tg = Td.cpu().numpy() if energy else None

    # end to end: host (pinned) buffers through the public API, copies timed
    e2e = None
    if not args.no_e2e:
        T0h = torch.as_tensor(T)
        Th = T0h.clone().pin_memory()
        ph = torch.as_tensor(p).pin_memory()
        Y0h = torch.as_tensor(Y0).contiguous()
        Yh = torch.empty_like(Y0h).pin_memory()
        sth = torch.empty(cells, dtype=torch.uint8).pin_memory()
        hbuf = kin.host_buffer(km, cells, method, prec, device=dev, sigma=sigma, energy=energy,
                               **shape)

        def e2e_step():
            # the flow solver hands over its state in host memory every step
            Yh.copy_(Y0h)
            if energy:
                Th.copy_(T0h)
            kin.integrate_host(km, Th, ph, Yh, w["dt"], w["rtol"], w["atol"], method, prec,
                               status=sth, buffer=hbuf, stream=stream, sigma=sigma,
                               energy=energy, **shape)
            stream.synchronize()

        e2e_step()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        ne = max(1, min(args.steps, 3))
        for _ in range(ne):
            e2e_step()
        el = time.perf_counter() - t0
        te = torch.tensor([el], device=dev, dtype=torch.float64)
        if world > 1:
            dist.all_reduce(te, op=dist.ReduceOp.MAX)
        e2e = {"value": world * cells_per_rank * ne / float(te.item()), "unit": UNIT,
               "h2d_bytes_per_step": int(Th.numel() * 8 + ph.numel() * 8 + Yh.numel() * 8),
               "d2h_bytes_per_step": int(Yh.numel() * 8 + sth.numel() + (Th.numel() * 8 if energy else 0)),
               "api": "kin_integrate_host (pinned host buffers)"}

    cpu = acc = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ref = {}
        v, nt, sample = oracle_rate(name, cells_target_s=args.cpu_seconds, max_cells=cells, result=ref,
                                    cells=cells, order=args.order)
        cpu = {"value": v, "unit": UNIT, "cores": nt, "kind": "oracle", "sample": sample}
        v1, _, sample1 = oracle_rate(name, cells_target_s=args.cpu_seconds / 2, nthreads=1)
        cpu["single_core"] = {"value": v1, "unit": UNIT, "cores": 1, "sample": sample1}
        # the GPU's own results on those cells (the last timed call) against
        # the oracle's: the error per result that the precision target names
        n = ref["n"]
        acc = accuracy(m, Yg[:, :n], ref["Y"], status[:n], ref["status"], stats[:n], ref["stats"],
                       w["atol"], w["rtol"], None if Tg is None else Tg[:n], ref["T"])
        acc["sample"] = "the cpu_baseline cells: " + sample

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == synth.FP64 else "f32+f64",
            "data": "synthetic (seeded generator standing in for the paper's mechanisms and states)",
            "config": dict(workload_config(name, cells_per_rank, sigma, args.order), launch_shape=shape,
                           f_evaluation=fname, cells_total=world * cells_per_rank,
                           parallelism="%d rank(s), one contiguous block of cells each "
                                       "(shard.shard_cells), no exchange" % world),
            "roofline": roof,
            "cpu_baseline": cpu,
            "accuracy_vs_oracle": acc,
            "e2e": e2e,
            "gpu_launches": args.steps * (5 if method == synth.RKC else
                                          (1 if layout_name(km, method, shape, cells) == "warp-per-cell"
                                           else 2)),
            "clocks": clk.summary(),
            "peak_probe": pk,
            "cell_status": np.bincount(status, minlength=4).tolist(),
            "mean_f_evals_per_cell": float(stats[:, 0].mean()),
            # the timed calls one by one (CUDA events around each kin_integrate,
            # excluding the L2 flush and the state reset between them)
            "call_ms": {"median": float(np.median(kern_ms)), "min": float(min(kern_ms)),
                        "max": float(max(kern_ms)), "n": len(kern_ms),
                        "cells_per_s_at_median": world * cells_per_rank / (float(np.median(kern_ms)) * 1e-3)},
        }
        if args.serve_requests > 0 and world == 1:
            line["serve"] = run_serve_leg(args)
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    km.close()
    return 0


def run_serve_leg(args):
    """The serving workload on this GPU: Poisson requests of 1,024-65,536
    cells (13-species FP64 or 53-species mixed, dt log-uniform 1e-7-1e-5 s),
    continuous batching against one launch per request at 0.8 of the
    saturated continuous-batching throughput, with p50/p99 latency and
    throughput of each (serve.benchmark), and the SM clocks sampled over it."""
    from paper_1309_2710_gb300 import serve
    n = args.serve_requests
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        out = serve.benchmark(requests=n, loads=(0.8,), saturation_requests=max(50, n // 2))
    out["clocks"] = clk.summary()
    out["workload"] = ("%d Poisson requests at 0.8 load (saturation measured on %d requests at t = 0); "
                       "continuous batching: %d slots per mechanism, per-launch cell caps %s; "
                       "latency = arrival to result in pinned host memory"
                       % (n, max(50, n // 2), out["slots_per_group"], out["batch_cells_cap"]))
    return out


# ------------------------------------------------------- batched mode ---
def run_batched(args):
    """The 16-instance 111-species workload: one persistent launch over all
    instances (replayed from a CUDA graph) against 16 separate launches."""
    import torch
    from paper_1309_2710_gb300 import build as kbuild
    kbuild.build()
    from paper_1309_2710_gb300 import kin
    name = "c2h4_111sp_rkc_batched"
    w = synth.WORKLOADS[name]
    m = synth.workload_mechanism(name)
    km = kin.Mechanism(m)
    prec = synth.MIXED if args.precision == "mixed" else synth.FP64
    dev = torch.device("cuda")
    inst = synth.batched_instances(name, scale=args.scale)
    parts, Y0s = [], []
    for i, (n, dt) in enumerate(inst):
        T, p, Y = synth.workload_states(name, m, cells=n, seed_offset=100 + i)
        Yd = torch.as_tensor(Y, device=dev).contiguous()
        Y0s.append(Yd.clone())
        parts.append(kin.Cells(torch.as_tensor(T, device=dev), torch.as_tensor(p, device=dev), Yd, dt,
                               w["rtol"], w["atol"], torch.zeros(n, dtype=torch.uint8, device=dev),
                               torch.zeros((n, kin.NSTATS), dtype=torch.int32, device=dev)))
    total = sum(n for n, _ in inst)
    sigma = w["sigma"] if args.sigma == "default" else (synth.POWER if args.sigma == "power"
                                                         else synth.GERSHGORIN)
    shape = dict(block_threads=0, blocks_per_sm=0, staging=kin.STAGE_GLOBAL, occupancy=kin.OCC_DEFAULT,
                 layout=kin.LAYOUT_AUTO)
    if args.shape:
        v = [int(x) for x in args.shape.split(",")]
        shape.update(zip(("block_threads", "blocks_per_sm", "staging", "occupancy", "layout"), v))
    elif not args.no_tune:
        # block shape from the autotuner, timed on a 16384-cell sample of the
        # mechanism's states (outside the timed region)
        from paper_1309_2710_gb300 import autotune
        Ts, ps, Ys = synth.workload_states(name, m, cells=16384, seed_offset=99)
        best = autotune.tune(km, m, torch.as_tensor(Ts, device=dev), torch.as_tensor(ps, device=dev),
                             torch.as_tensor(Ys, device=dev).contiguous(), inst[0][1], w["rtol"],
                             w["atol"], kin.RKC, prec, sigma=sigma)
        shape = {k: best[k] for k in shape}
    ws = km.workspace(kin.RKC, prec, total, shape["block_threads"], shape["blocks_per_sm"], dev,
                      shape["staging"], shape["occupancy"], sigma, shape["layout"])
    ws1 = km.workspace(kin.RKC, prec, max(n for n, _ in inst), shape["block_threads"],
                       shape["blocks_per_sm"], dev, shape["staging"], shape["occupancy"], sigma,
                       shape["layout"])
    stream = torch.cuda.Stream()

    def reset():
        for c, y0 in zip(parts, Y0s):
            c.Y.copy_(y0)

    def separate():
        for c in parts:
            kin.integrate(km, c.T, c.p, c.Y, c.dt, c.rtol, c.atol, kin.RKC, prec, status=c.status,
                          stats=c.stats, workspace=ws1, stream=stream, sigma=sigma, **shape)

    with torch.cuda.stream(stream):
        reset()
        kin.integrate_batch(km, parts, kin.RKC, prec, workspace=ws, stream=stream, sigma=sigma, **shape)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        kin.integrate_batch(km, parts, kin.RKC, prec, workspace=ws, sigma=sigma, **shape)
    out = {}
    pk = measure_peaks(torch.cuda.current_device())
    for label, fn in (("persistent_graph", g.replay), ("separate_launches", separate)):
        for _ in range(args.warmup):
            with torch.cuda.stream(stream):
                reset()
                fn()
        torch.cuda.synchronize()
        ms = []
        with ClockSampler(torch.cuda.current_device()) as clk:
            for _ in range(args.steps):
                with torch.cuda.stream(stream):
                    reset()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    fn()
                    e1.record(stream)
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
        st = torch.cat([c.status for c in parts]).cpu().numpy()
        out[label] = {"ms": float(np.median(ms)), "cells_per_s": total / (np.median(ms) * 1e-3),
                      "status": np.bincount(st, minlength=4).tolist(), "clocks": clk.summary()}
    stats = torch.cat([c.stats for c in parts]).cpu().numpy()
    nfe = float(stats[:, 0].mean())
    roof = roofline(m, synth.RKC, prec, sigma, stats, 0, out["persistent_graph"]["ms"], pk)
    cpu = None if args.no_cpu_baseline else oracle_batched_sample(name, m, inst, args.stage_sample)
    print(json.dumps({"mode": "batched", "workload": name, "instances": len(inst), "cells": total,
                      "cpu_baseline": cpu, "gpu_f_evals_per_cell": {
                          "min": int(stats[:, 0].min()), "median": float(np.median(stats[:, 0])),
                          "max": int(stats[:, 0].max())},
                      "scale": args.scale, "precision": args.precision, "mean_f_evals": nfe,
                      "sigma": "power" if sigma == synth.POWER else "gershgorin",
                      "sizes": [n for n, _ in inst], "launch_shape": shape, **out, "roofline": roof,
                      "speedup": out["separate_launches"]["ms"] / out["persistent_graph"]["ms"]}))
    return 0


def oracle_batched_sample(name, m, inst, per_dt):
    """The CPU leg of the batched line: the FP64 oracle on a bounded sample
    of the batched workload, `per_dt` cells for each dt (taken in turn from
    the instances with that dt, the same states as the GPU run), timed on the
    host cores, with the RKC stage count of every attempt traced: the
    workload's stiffness spread that the persistent launch balances."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    w = synth.WORKLOADS[name]
    om = oracle.Mech(m)
    sample, stages = [], {}
    for dt in sorted(set(d for _, d in inst)):
        picks = [(i, n) for i, (n, d) in enumerate(inst) if d == dt]
        states = [synth.workload_states(name, m, cells=n, seed_offset=100 + i) for i, n in picks]
        cells, k = [], 0
        while len(cells) < per_dt and k < max(n for _, n in picks):
            for j, (i, n) in enumerate(picks):
                if k < n and len(cells) < per_dt:
                    T, p, Y = states[j]
                    cells.append((T[k], p[k], Y[:, k].copy()))
            k += 1
        sample.append((dt, cells))
    threads = os.cpu_count() or 1

    def one(args):
        dt, (T, p, y) = args
        _, st, tr = oracle.trace_cell(om, T, p, y, dt, w["rtol"], w["atol"], oracle_method(w), cap=200000)
        return dt, st, tr["s"], int(tr["stats"][0])

    jobs = [(dt, c) for dt, cells in sample for c in cells]
    t0 = time.perf_counter()
    with ThreadPoolExecutor(threads) as ex:  # the oracle's C code runs without the GIL
        res = list(ex.map(one, jobs))
    el = time.perf_counter() - t0
    for dt in sorted(set(r[0] for r in res)):
        rr = [r for r in res if r[0] == dt]
        s_all = np.concatenate([r[2] for r in rr])
        smax = np.array([r[2].max() for r in rr])
        nfe = np.array([r[3] for r in rr])
        stages["%g" % dt] = {
            "cells": len(rr), "status": np.bincount([r[1] for r in rr], minlength=4).tolist(),
            "stages_per_attempt": {"min": int(s_all.min()), "p50": float(np.percentile(s_all, 50)),
                                   "p90": float(np.percentile(s_all, 90)), "p99": float(np.percentile(s_all, 99)),
                                   "max": int(s_all.max())},
            "max_stages_per_cell": {"min": int(smax.min()), "p50": float(np.median(smax)), "max": int(smax.max())},
            "f_evals_per_cell": {"min": int(nfe.min()), "p50": float(np.median(nfe)), "max": int(nfe.max())},
            "histogram_stages_by_25": np.bincount(np.minimum(s_all, 250) // 25, minlength=11).tolist()}
    return {"value": len(jobs) / el, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": "%d cells per dt, the first cells of the instances with that dt in turn, %.1f s wall"
                      % (per_dt, el), "stage_counts": stages}


def run_divergence(args):
    """The divergence study of Section 3.1: `--global-steps` consecutive calls
    (flow steps) on the same cells, 65,536 by default as in the paper, once
    with the cells in 'similar' order (sorted by temperature) and once as
    drawn ('random'). Reports each order's time and the distribution of the
    warp divergence measure D over the per-cell f evaluations summed over the
    calls, for the paper's fixed thread-per-cell mapping and for the best
    fixed mapping (cells sorted by count)."""
    import torch
    from paper_1309_2710_gb300 import build as kbuild
    from paper_1309_2710_gb300 import divergence
    kbuild.build()
    from paper_1309_2710_gb300 import kin
    name = args.workload
    w = synth.WORKLOADS[name]
    m = synth.workload_mechanism(name)
    km = kin.Mechanism(m)
    cells = args.cells or 65536
    dev = torch.device("cuda")
    method, prec = w["method"], w["precision"]
    sigma = w["sigma"] if args.sigma == "default" else (synth.POWER if args.sigma == "power"
                                                         else synth.GERSHGORIN)
    energy = int(bool(w.get("energy")))
    states = {o: synth.workload_states(name, m, cells=cells, sort_by_T=o == "similar")
              for o in ("similar", "random")}
    shape = dict(block_threads=0, blocks_per_sm=0, staging=kin.STAGE_GLOBAL, occupancy=kin.OCC_DEFAULT,
                 layout=kin.LAYOUT_AUTO)
    if args.shape:
        v = [int(x) for x in args.shape.split(",")]
        shape.update(zip(("block_threads", "blocks_per_sm", "staging", "occupancy", "layout"), v))
    elif not args.no_tune:
        from paper_1309_2710_gb300 import autotune
        T, p, Y = states["random"]
        best = autotune.tune(km, m, torch.as_tensor(T, device=dev), torch.as_tensor(p, device=dev),
                             torch.as_tensor(Y, device=dev).contiguous(), w["dt"], w["rtol"],
                             w["atol"], method, prec, sigma=sigma, energy=energy)
        shape = {k: best[k] for k in shape}
    ws = km.workspace(method, prec, cells, shape["block_threads"], shape["blocks_per_sm"], dev,
                      shape["staging"], shape["occupancy"], sigma, shape["layout"], energy)
    stream = torch.cuda.current_stream()
    st = torch.zeros(cells, dtype=torch.uint8, device=dev)
    sta = torch.zeros((cells, kin.NSTATS), dtype=torch.int32, device=dev)
    out = {}
    for order, (T, p, Y) in states.items():
        T0d, pd = torch.as_tensor(T, device=dev), torch.as_tensor(p, device=dev)
        Y0d = torch.as_tensor(Y, device=dev).contiguous()
        Td, Yd = T0d.clone(), Y0d.clone()

        def call():
            kin.integrate(km, Td, pd, Yd, w["dt"], w["rtol"], w["atol"], method, prec, status=st,
                          stats=sta, workspace=ws, stream=stream, sigma=sigma, energy=energy, **shape)

        for _ in range(args.warmup):
            call()
        Td.copy_(T0d)
        Yd.copy_(Y0d)
        torch.cuda.synchronize()
        d = np.zeros(cells, dtype=np.int64)
        ms, bad = [], 0
        for _ in range(args.global_steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            call()
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
            d += sta[:, 0].cpu().numpy()
            bad += int((st != 0).sum().item())
        out[order] = {"ms_total": float(sum(ms)), "ms_per_call": [float(x) for x in ms],
                      "cells_per_s": cells * len(ms) / (sum(ms) * 1e-3), "nonzero_status": bad,
                      "mean_f_evals_per_call": float(d.mean() / len(ms)),
                      "D": divergence.summary(d)}
    print(json.dumps({"mode": "divergence", "workload": name, "cells": cells,
                      "global_steps": args.global_steps, "launch_shape": shape,
                      "layout": layout_name(km, method, shape, cells),
                      "similar_over_random_time": out["similar"]["ms_total"] / out["random"]["ms_total"],
                      **out}))
    km.close()
    return 0


def feval_name(km, prec, shape, cells, layout, energy=0):
    """'generated' where the call runs the generated f (asked for, or the
    library's automatic choice: lane layout, FP64, isothermal, staging 0, a
    small mechanism, a large call), else 'tables'."""
    from paper_1309_2710_gb300 import kin
    if shape.get("feval", kin.FEVAL_AUTO) != kin.FEVAL_AUTO:
        return "generated" if shape["feval"] == kin.FEVAL_GENERATED else "tables"
    gen = (layout == "lane-per-cell" and prec == synth.FP64 and not energy
           and shape.get("staging", 0) == kin.STAGE_GLOBAL and km.n_species <= kin.GEN_MAX_SPECIES
           and km.n_reactions <= kin.GEN_MAX_REACTIONS and cells >= kin.GEN_MIN_CELLS)
    return "generated" if gen else "tables"


def layout_name(km, method, shape, cells):
    from paper_1309_2710_gb300 import kin
    import torch
    lay = shape.get("layout", kin.LAYOUT_AUTO)
    if lay == kin.LAYOUT_AUTO:
        nsm = torch.cuda.get_device_properties(0).multi_processor_count
        small = cells < kin.WARP_MAX_CELLS_PER_SM * nsm
        lay = kin.LAYOUT_WARP if km.n_reactions > kin.WARP_MIN_REACTIONS or small else kin.LAYOUT_LANE
    return "warp-per-cell" if lay == kin.LAYOUT_WARP else "lane-per-cell"


def launcher_cmd(argv, n_gpus, port):
    """The command that runs this benchmark as n_gpus ranks on one node,
    one process per GPU (rendezvous on 127.0.0.1)."""
    return [sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
            "--nproc-per-node", str(n_gpus), "--master-addr", "127.0.0.1", "--master-port", str(port),
            os.path.abspath(__file__)] + list(argv)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["kin", "reference"], default="kin")
    ap.add_argument("--workload", default="h2co_13sp_rkc", choices=[k for k, v in synth.WORKLOADS.items()
                                                                   if v["cells"]])
    ap.add_argument("--cells", type=int, default=0)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="library default launch shape")
    ap.add_argument("--shape", default="", help="block_threads,blocks_per_sm,staging,occupancy"
                                                "[,layout] (skips the autotuner)")
    ap.add_argument("--mode", choices=["headline", "batched", "divergence"], default="headline")
    ap.add_argument("--global-steps", type=int, default=10,
                    help="divergence mode: consecutive calls whose f evaluations are summed")
    ap.add_argument("--order", choices=["random", "sorted"], default="random",
                    help="cell order: as drawn, or sorted by temperature ('similar')")
    ap.add_argument("--sigma", choices=["default", "gershgorin", "power"], default="default",
                    help="RKC spectral-radius estimator (default: the workload's)")
    ap.add_argument("--scale", type=float, default=1.0, help="batched mode: instance size scale")
    ap.add_argument("--feval", choices=["auto", "table", "generated"], default="auto",
                    help="f evaluation of the lane layout (default: the library's choice)")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64",
                    help="batched mode: rate precision")
    ap.add_argument("--serve-requests", type=int, default=300,
                    help="requests of the serving leg on the headline line (0: no serving leg)")
    ap.add_argument("--stage-sample", type=int, default=96,
                    help="batched mode: cells per dt whose RKC stage counts the oracle traces")
    args = ap.parse_args()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        # one process per GPU: re-run this command under torch.distributed.run
        import socket
        with socket.socket() as sk:
            sk.bind(("127.0.0.1", 0))
            port = sk.getsockname()[1]
        return subprocess.call(launcher_cmd(sys.argv[1:], args.gpus, port))
    if args.mode == "batched":
        return run_batched(args)
    if args.mode == "divergence":
        return run_divergence(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_kin(args)


if __name__ == "__main__":
    sys.exit(main())
