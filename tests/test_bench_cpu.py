"""Host logic of the benchmark on the CPU: the algorithmic operation count
behind the roofline fraction, the f-evaluation label and the DRAM traffic
lookup."""
import types

import numpy as np

import bench
from paper_1309_2710_gb300 import synth
from tests import mechs


def small_mech():
    # 3 species: A -> B (1 reactant), A + B -> C (2), third body A + C -> 2 B
    # (2 reactants, [M] over 3 species), falloff C -> A (1 reactant)
    m = mechs.mech([2.0, 3.0, 5.0],
                   [dict(reac=[0], prod=[1], A=1.0),
                    dict(reac=[0, 1], prod=[2], A=1.0),
                    dict(reac=[0, 2], prod=[1, 1], A=1.0, type=1),
                    dict(reac=[2], prod=[0], A=1.0, type=2, A0=2.0)],
                   eff_rows=[[1.0, 1.0, 1.0], [1.0, 1.0, 1.0]])
    m.n_species, m.n_reactions = 3, 4
    return m


def test_feval_ops_by_hand():
    m = small_mech()
    nS = 3
    mixture = 3 * nS + 1
    reactants = 1 + 2 + 2 + 1
    third_body = nS + 1
    falloff = nS + 4
    # net nonzeros: r0 A,B; r1 A,B,C; r2 A,B,C; r3 C,A
    nonzeros = 2 + 3 + 3 + 2
    scaling = nS + 1
    assert bench.feval_ops(m) == mixture + reactants + third_body + falloff + nonzeros + scaling


def test_feval_ops_of_the_workload_mechanisms():
    got = [bench.feval_ops(synth.workload_mechanism(n))
           for n in ("h2_9sp_rkck", "h2co_13sp_rkc", "ch4_53sp_rkc_mixed", "c2h4_111sp_rkc_batched")]
    assert got == [256, 440, 8160, 31050]


def stats(rows):
    return np.asarray(rows, dtype=np.int32).reshape(-1, 5)


def test_algorithmic_work_rkck():
    m = small_mech()
    f = bench.feval_ops(m)
    st = stats([[60, 8, 2, 0, 0], [30, 5, 0, 0, 0]])
    o64, o32, exact = bench.algorithmic_work(m, synth.RKCK, synth.FP64, synth.GERSHGORIN, st)
    assert exact and o32 == 0
    assert o64 == (60 + 30) * f + (10 + 5) * 38 * 3


def test_algorithmic_work_rkc_gershgorin_and_mixed_split():
    m = small_mech()
    nS, f = 3, bench.feval_ops(m)
    # one cell: 40 f evaluations, 6 of them in 2 Gershgorin estimates (3 columns each),
    # 10 accepted + 1 rejected attempts
    st = stats([[40, 10, 1, 2, 6]])
    o64, o32, exact = bench.algorithmic_work(m, synth.RKC, synth.FP64, synth.GERSHGORIN, st)
    rate = 40 - 6
    stages = rate - 2
    vec = (stages - 11) * 5 * nS + 11 * 8 * nS + 6 * 3 * nS + 6 * nS
    assert exact and o32 == 0 and o64 == 40 * f + vec
    # mixed: rate evaluations keep only the final scaling in FP64; the sigma
    # evaluations (here the power method, which adds an FP64 base evaluation
    # per estimate) stay FP64
    st = stats([[40, 10, 1, 2, 8]])
    o64, o32, exact = bench.algorithmic_work(m, synth.RKC, synth.MIXED, synth.POWER, st)
    rate = 40 - 8
    stages = rate - 2
    vec = (stages - 11) * 5 * nS + 11 * 8 * nS + (8 - 2) * 4 * nS + 6 * nS
    assert exact
    assert o32 == rate * (f - (nS + 1))
    assert o64 == rate * (nS + 1) + 8 * f + vec


def test_energy_count_is_a_lower_bound():
    m = synth.workload_mechanism("h2co_13sp_rkc_energy")
    st = stats([[30, 5, 0, 1, 4]])
    _, _, exact = bench.algorithmic_work(m, synth.RKC, synth.FP64, synth.POWER, st, energy=True)
    assert not exact


def test_feval_label():
    km = types.SimpleNamespace(n_species=13, n_reactions=54)
    big = types.SimpleNamespace(n_species=53, n_reactions=634)
    lane, warp = "lane-per-cell", "warp-per-cell"
    sh = dict(staging=0)
    assert bench.feval_name(km, synth.FP64, sh, 262144, lane) == "generated"
    assert bench.feval_name(km, synth.FP64, sh, 1000, lane) == "tables"
    assert bench.feval_name(km, synth.MIXED, sh, 262144, lane) == "tables"
    assert bench.feval_name(km, synth.FP64, sh, 262144, warp) == "tables"
    assert bench.feval_name(km, synth.FP64, dict(staging=1), 262144, lane) == "tables"
    assert bench.feval_name(km, synth.FP64, sh, 262144, lane, energy=1) == "tables"
    assert bench.feval_name(big, synth.FP64, sh, 262144, lane) == "tables"
    assert bench.feval_name(km, synth.FP64, dict(staging=0, feval=2), 10, lane) == "generated"
    assert bench.feval_name(km, synth.FP64, dict(staging=0, feval=1), 262144, lane) == "tables"


def test_traffic_lookup(monkeypatch):
    monkeypatch.setattr(bench, "kernel_hash", lambda: "h")
    monkeypatch.setattr(bench, "TRAFFIC", {"h": {("w", (32, 16, 0, 0, 1), "generated"): (100.0, 10),
                                                 ("w", (32, 20, 0, 1, 1), "generated"): (300.0, 10)}})
    # exact shape, scaled by cells
    assert bench.traffic_for("w", (32, 16, 0, 0, 1), "generated", 20) == (200.0, [32, 16, 0, 0, 1])
    # same kernel variant and resident lanes per SM
    assert bench.traffic_for("w", (128, 4, 0, 0, 1), "generated", 10) == (100.0, [32, 16, 0, 0, 1])
    # another register budget, another f, another workload or other sources: none
    assert bench.traffic_for("w", (128, 4, 0, 1, 1), "generated", 10) == (None, None)
    assert bench.traffic_for("w", (32, 16, 0, 0, 1), "tables", 10) == (None, None)
    assert bench.traffic_for("v", (32, 16, 0, 0, 1), "generated", 10) == (None, None)
    monkeypatch.setattr(bench, "kernel_hash", lambda: "other")
    assert bench.traffic_for("w", (32, 16, 0, 0, 1), "generated", 10) == (None, None)


def test_contract_flops_by_hand():
    """The hot-path contract's flop count: per f evaluation
    F = 4 nS + 2 nR + 2 nS nM + 6 nFO + 8 nR + 2 nS; RKC adds 10 nS per
    stage, 14 nS per attempt, 2 nS^2 per spectral-radius estimate."""
    m = small_mech()  # nS 3, nR 4, nM 2, nFO 1
    F = 4 * 3 + 2 * 4 + 2 * 3 * 2 + 6 * 1 + 8 * 4 + 2 * 3
    assert F == 76
    st = stats([[40, 10, 1, 2, 6]])
    f64, f32 = bench.contract_flops(m, synth.RKC, synth.FP64, st)
    stages, att = 40 - 6 - 2, 11
    assert f32 == 0
    assert f64 == 34 * F + stages * 10 * 3 + att * 14 * 3 + 2 * 2 * 9 + 6 * F
    st = stats([[40, 10, 1, 2, 8]])
    f64, f32 = bench.contract_flops(m, synth.RKC, synth.MIXED, st)
    rate = 40 - 8
    assert f32 == rate * (F - 2 * 3)
    assert f64 == rate * 2 * 3 + (rate - 2) * 10 * 3 + att * 14 * 3 + 2 * 2 * 9 + 8 * F
    st = stats([[60, 8, 2, 0, 0]])
    f64, f32 = bench.contract_flops(m, synth.RKCK, synth.FP64, st)
    assert f64 == 60 * F + 10 * 60 * 3 and f32 == 0


def test_contract_flops_per_evaluation_of_the_headline_mechanism():
    # 13 species, 54 reactions, 5 third-body reactions, no falloff: 748 flops
    m = synth.workload_mechanism("h2co_13sp_rkc")
    assert bench.contract_flops(m, synth.RKCK, synth.FP64, stats([[1, 0, 0, 0, 0]]))[0] == 748


def test_launcher_runs_one_process_per_gpu():
    cmd = bench.launcher_cmd(["--gpus", "4", "--steps", "3"], 4, 29511)
    assert cmd[1:3] == ["-m", "torch.distributed.run"]
    i = cmd.index("--nproc-per-node")
    assert cmd[i + 1] == "4"
    assert cmd[cmd.index("--master-addr") + 1] == "127.0.0.1"
    assert cmd[cmd.index("--master-port") + 1] == "29511"
    assert cmd[-4:] == ["--gpus", "4", "--steps", "3"] and cmd[-5].endswith("bench.py")
