"""GPU parity of the warp-per-cell layout (one warp integrates one cell; the
library's choice for RKC mechanisms above 256 reactions) against the FP64
oracle, on every register-vector width (1, 2, 4 and 8 slots of 32 species),
both spectral-radius estimators and both rate precisions, plus the
properties the layout must share with the lane-per-cell kernel."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1309_2710_gb300 import synth  # noqa: E402
from tests.oracle_variants import reference  # noqa: E402
from tests.parity import compare, compare_mixed, rel_err, tol_rel_err  # noqa: E402

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1309_2710_gb300 import build as kbuild  # noqa: E402

kbuild.build()
from paper_1309_2710_gb300 import kin  # noqa: E402

DEV = torch.device("cuda:0")
WARP = kin.LAYOUT_WARP
_MECHS = {}

# 140 species fill 8 register slots per lane (species l + 32 r, r < 5 used)
WIDE = dict(n_species=140, n_reactions=300, elements=("H", "O", "C", "N"), tb_frac=0.1,
            fo_frac=0.05, seed=77)


def mech(name):
    if name not in _MECHS:
        if name == "wide_140sp":
            m = synth.make_mechanism(**WIDE)
        else:
            m = synth.workload_mechanism(name)
        _MECHS[name] = (m, kin.Mechanism(m), oracle.Mech(m))
    return _MECHS[name]


def states(name, m, cells, seed):
    if name == "wide_140sp":
        return synth.make_states(m, cells, T_range=(900.0, 1800.0), seed=seed)
    return synth.workload_states(name, m, cells=cells, seed_offset=seed)


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device=DEV)


def run(km, T, p, Y, dt, precision=kin.FP64, sigma=kin.SIGMA_GERSHGORIN, layout=WARP,
        max_steps=20000, ld=None, **shape):
    cells = T.shape[0]
    ld = cells if ld is None else ld
    Yd = torch.zeros((Y.shape[0], ld), dtype=torch.float64, device=DEV)
    Yd[:, :cells] = dev(Y)
    st = torch.full((cells,), 255, dtype=torch.uint8, device=DEV)
    sta = torch.zeros((cells, kin.NSTATS), dtype=torch.int32, device=DEV)
    kin.integrate(km, dev(T), dev(p), Yd, dt, 1e-6, 1e-10, kin.RKC, precision, status=st,
                  stats=sta, max_steps=max_steps, sigma=sigma, layout=layout, **shape)
    torch.cuda.synchronize()
    return Yd.cpu().numpy(), st.cpu().numpy(), sta.cpu().numpy()


def oracle_method(sigma):
    return oracle.RKC_POWER if sigma == kin.SIGMA_POWER else oracle.RKC


@pytest.mark.parametrize("name,cells,sigma", [
    ("h2co_13sp_rkc", 1, kin.SIGMA_GERSHGORIN),          # 1 slot, a single cell
    ("h2co_13sp_rkc", 777, kin.SIGMA_GERSHGORIN),
    ("h2co_13sp_rkc", 333, kin.SIGMA_POWER),
    ("ch4_53sp_rkc_mixed", 33, kin.SIGMA_GERSHGORIN),    # 2 slots
    ("ch4_53sp_rkc_mixed", 301, kin.SIGMA_POWER),
    ("c2h4_111sp_rkc_batched", 40, kin.SIGMA_POWER),     # 4 slots
    ("wide_140sp", 37, kin.SIGMA_GERSHGORIN),            # 8 slots
    ("wide_140sp", 37, kin.SIGMA_POWER),
])
def test_warp_fp64_against_oracle(name, cells, sigma):
    m, km, om = mech(name)
    T, p, Y = states(name, m, cells, 31)
    dt = 1e-6
    Yg, stg, stag = run(km, T, p, Y, dt, sigma=sigma, ld=cells + 3)
    Yo, sto, stao, fl = reference(m, T, p, Y, dt, 1e-6, 1e-10, oracle_method(sigma))
    frac = 0.05 if sigma == kin.SIGMA_POWER else 0.01
    s = compare(Yg[:, :cells], Yo, stg, sto, stag, stao, 1e-10, 1e-6,
                max_div_frac=max(frac, 1.0 / cells), floor=fl)
    assert np.all(Yg[:, cells:] == 0.0)  # padding columns untouched
    print("warp fp64", name, cells, sigma, s)


@pytest.mark.parametrize("sigma", [kin.SIGMA_GERSHGORIN, kin.SIGMA_POWER])
def test_warp_mixed_ch4(sigma):
    """FP32 rates, FP64 state: two valid RKC solutions, compared per species
    at the integrator's own weighting (as for the lane layout)."""
    name = "ch4_53sp_rkc_mixed"
    m, km, om = mech(name)
    T, p, Y = states(name, m, 1024, 32)
    Yg, stg, stag = run(km, T, p, Y, 1e-6, precision=kin.MIXED, sigma=sigma)
    idx = np.arange(0, 1024, 8)
    Yo, sto, stao, _ = oracle.integrate(om, T[idx], p[idx], Y[:, idx], 1e-6, 1e-6, 1e-10,
                                        oracle_method(sigma))
    print("warp mixed ch4", sigma, compare_mixed(Yg[:, idx], Yo, stg[idx], sto, stag[idx], stao, 1e-10, 1e-6))


def test_warp_mixed_c2h4():
    name = "c2h4_111sp_rkc_batched"
    m, km, om = mech(name)
    T, p, Y = states(name, m, 512, 33)
    Yg, stg, stag = run(km, T, p, Y, 1e-6, precision=kin.MIXED, sigma=kin.SIGMA_POWER)
    idx = np.arange(0, 512, 16)
    Yo, sto, stao, _ = oracle.integrate(om, T[idx], p[idx], Y[:, idx], 1e-6, 1e-6, 1e-10,
                                        oracle.RKC_POWER)
    print("warp mixed c2h4", compare_mixed(Yg[:, idx], Yo, stg[idx], sto, stag[idx], stao, 1e-10, 1e-6))


def test_warp_and_lane_layouts_agree():
    """Same method and decisions: statuses equal, decision traces equal on
    nearly every cell, states within the parity tolerance."""
    name = "ch4_53sp_rkc_mixed"
    m, km, om = mech(name)
    T, p, Y = states(name, m, 600, 34)
    Yw, sw, xw = run(km, T, p, Y, 1e-6, layout=WARP)
    Yl, sl, xl = run(km, T, p, Y, 1e-6, layout=kin.LAYOUT_LANE)
    s = compare(Yw, Yl, sw, sl, xw, xl, 1e-10, 1e-6)
    print("warp vs lane", s)


def test_auto_layout_picks_warp_above_threshold():
    name = "ch4_53sp_rkc_mixed"
    m, km, om = mech(name)
    assert m.n_reactions > kin.WARP_MIN_REACTIONS
    T, p, Y = states(name, m, 200, 35)
    Ya, sa, xa = run(km, T, p, Y, 1e-6, layout=kin.LAYOUT_AUTO)
    Yw, sw, xw = run(km, T, p, Y, 1e-6, layout=WARP)
    assert np.array_equal(Ya, Yw) and np.array_equal(xa, xw)


@pytest.mark.parametrize("precision", [kin.FP64, kin.MIXED])
def test_warp_launch_shapes_are_bitwise_identical(precision):
    """A cell's arithmetic does not depend on which warp, block or SM takes it."""
    name = "ch4_53sp_rkc_mixed"
    m, km, om = mech(name)
    T, p, Y = states(name, m, 1000, 36)
    ref = None
    for shape in [dict(), dict(block_threads=256, blocks_per_sm=1),
                  dict(block_threads=64, blocks_per_sm=2), dict(block_threads=32, blocks_per_sm=1)]:
        Yg, sg, xg = run(km, T, p, Y, 1e-6, precision=precision, sigma=kin.SIGMA_POWER, **shape)
        if ref is None:
            ref = (Yg, sg, xg)
        else:
            assert np.array_equal(Yg, ref[0]) and np.array_equal(xg, ref[2]), shape


def test_warp_batch_equals_separate_calls():
    name = "c2h4_111sp_rkc_batched"
    m, km, om = mech(name)
    parts, singles = [], []
    for i, (n, dt) in enumerate([(70, 1e-6), (5, 1e-5), (130, 3e-6), (1, 1e-6)]):
        T, p, Y = states(name, m, n, 40 + i)
        parts.append(kin.Cells(dev(T), dev(p), dev(Y), dt))
        Ys = dev(Y)
        kin.integrate(km, dev(T), dev(p), Ys, dt, 1e-6, 1e-10, kin.RKC, kin.MIXED,
                      sigma=kin.SIGMA_POWER, layout=WARP)
        singles.append(Ys)
    kin.integrate_batch(km, parts, kin.RKC, kin.MIXED, sigma=kin.SIGMA_POWER, layout=WARP)
    torch.cuda.synchronize()
    for c, Ys in zip(parts, singles):
        assert torch.equal(c.Y, Ys)


def test_warp_batch_in_cuda_graph():
    name = "ch4_53sp_rkc_mixed"
    m, km, om = mech(name)
    host = [states(name, m, n, 50 + i) for i, n in enumerate([300, 9, 700])]
    parts = [kin.Cells(dev(T), dev(p), dev(Y), 1e-6, 1e-6, 1e-10,
                       torch.zeros(len(T), dtype=torch.uint8, device=DEV)) for T, p, Y in host]
    Y0 = [c.Y.clone() for c in parts]
    ws = km.workspace(kin.RKC, kin.MIXED, 1009, sigma=kin.SIGMA_POWER, layout=WARP)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        kin.integrate_batch(km, parts, kin.RKC, kin.MIXED, workspace=ws, sigma=kin.SIGMA_POWER,
                            layout=WARP)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    eager = [c.Y.clone() for c in parts]
    for c, y0 in zip(parts, Y0):
        c.Y.copy_(y0)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        kin.integrate_batch(km, parts, kin.RKC, kin.MIXED, workspace=ws, sigma=kin.SIGMA_POWER,
                            layout=WARP)
    for _ in range(2):
        for c, y0 in zip(parts, Y0):
            c.Y.copy_(y0)
        g.replay()
        torch.cuda.synchronize()
        for c, e in zip(parts, eager):
            assert torch.equal(c.Y, e)
            assert int(c.status.max()) == 0


def test_warp_step_limit_and_nonfinite_cell():
    name = "ch4_53sp_rkc_mixed"
    m, km, om = mech(name)
    T, p, Y = states(name, m, 45, 37)
    Y[4, 9] = np.inf
    Yg, stg, stag = run(km, T, p, Y, 1e-6, max_steps=3)
    Yo, sto, stao, _ = oracle.integrate(om, T, p, Y, 1e-6, 1e-6, 1e-10, oracle.RKC, max_steps=3)
    assert stg[9] == kin.CELL_NONFINITE
    assert np.array_equal(stg, sto)
    assert np.isinf(Yg[4, 9])  # Y of a cell stopped by the pre-pass stays as given
    keep = np.arange(45) != 9
    # truncated runs: exact decision trace, state at the divergent tolerance
    # (see the lane-layout step-limit test for why)
    assert (stag[keep] == stao[keep]).all()
    compare(Yg[:, keep], Yo[:, keep], stg[keep], sto[keep], stag[keep], stao[keep], 1e-10, 1e-6,
            tol=1e-5)


def test_warp_zero_cells_and_bad_block_size():
    name = "ch4_53sp_rkc_mixed"
    m, km, om = mech(name)
    Y = torch.ones((m.n_species, 4), dtype=torch.float64, device=DEV)
    e = torch.empty(0, dtype=torch.float64, device=DEV)
    kin.integrate(km, e, e, Y, 1e-6, 1e-6, 1e-10, kin.RKC, layout=WARP)
    kin.integrate(km, e, e, Y, 1e-6, 1e-6, 1e-10, kin.RKCK, layout=WARP)
    torch.cuda.synchronize()
    assert torch.all(Y == 1)
    T, p, Yh = states(name, m, 4, 38)
    with pytest.raises(kin.KinError) as ex:
        kin.integrate(km, dev(T), dev(p), dev(Yh), 1e-6, 1e-6, 1e-10, kin.RKC, layout=WARP,
                      block_threads=512)
    assert ex.value.code == kin.KIN_EINVAL


def test_warp_full_size_ch4_sampled():
    """The 131072-cell, 53-species workload in the benchmark's configuration
    (mixed precision, power-method sigma, library launch shape); the oracle
    recomputes 8192 random cells; every cell conserves mass.

    FP32 rates perturb every error estimate a little, so on some cells the
    mixed path takes another accept/reject decision than the FP64 oracle (an
    extra rejection, say): a second valid RKC solution, one decision apart.
    As for trace-divergent FP64 cells, the target holds on the cells whose
    decisions (accepted and rejected step counts) equal the oracle's: 1e-5
    in the integrator's weighting. The others are held to the spread of valid
    rtol 1e-6 solutions, 1e-4 (the oracle's own result differs from a
    converged one by up to 8.8e-5); measured, up to 2.1e-5 on 32,768 cells."""
    name = "ch4_53sp_rkc_mixed"
    w = synth.WORKLOADS[name]
    m, km, om = mech(name)
    T, p, Y = synth.workload_states(name, m)
    Yg, stg, stag = run(km, T, p, Y, w["dt"], precision=kin.MIXED, sigma=kin.SIGMA_POWER,
                        layout=kin.LAYOUT_AUTO)
    idx = np.sort(np.random.default_rng(19).choice(T.shape[0], 8192, replace=False))
    Yo, sto, stao, _ = oracle.integrate(om, T[idx], p[idx], Y[:, idx], w["dt"], w["rtol"],
                                        w["atol"], oracle.RKC_POWER)
    assert (stg == 0).all()
    assert (sto == 0).all()
    print("warp full ch4 mixed", compare_mixed(Yg[:, idx], Yo, stg[idx], sto, stag[idx], stao, w["atol"],
                                                w["rtol"]))
    print("mass drift %.2e" % np.abs(Yg.sum(0) - 1).max())
    assert np.abs(Yg.sum(0) - 1).max() < 1e-7


# ------------------------------------------------------------------- RKCK ---
@pytest.mark.parametrize("name,cells,precision", [
    ("h2_9sp_rkck", 4096, kin.FP64),       # the full 9-species workload, 1 slot
    ("ch4_53sp_rkc_mixed", 77, kin.FP64),  # 2 slots
    ("wide_140sp", 19, kin.FP64),          # 8 slots
])
def test_warp_rkck_against_oracle(name, cells, precision):
    """Cash-Karp with one warp per cell (one persistent kernel, no pre-pass)."""
    m, km, om = mech(name)
    T, p, Y = states(name, m, cells, 71)
    dt = 1e-7
    Yd = dev(Y)
    st = torch.full((cells,), 255, dtype=torch.uint8, device=DEV)
    sta = torch.zeros((cells, kin.NSTATS), dtype=torch.int32, device=DEV)
    kin.integrate(km, dev(T), dev(p), Yd, dt, 1e-6, 1e-10, kin.RKCK, precision, status=st,
                  stats=sta, layout=WARP)
    torch.cuda.synchronize()
    Yo, sto, stao, fl = reference(m, T, p, Y, dt, 1e-6, 1e-10, oracle.RKCK)
    s = compare(Yd.cpu().numpy(), Yo, st.cpu().numpy(), sto, sta.cpu().numpy(), stao, 1e-10, 1e-6,
                floor=fl)
    print("warp rkck", name, cells, s)


def test_small_calls_choose_the_warp_layout():
    """Fewer cells than KIN_WARP_MAX_CELLS_PER_SM per SM: the automatic layout is
    one warp per cell (bit-identical to asking for it)."""
    name = "h2_9sp_rkck"
    m, km, om = mech(name)
    T, p, Y = states(name, m, 4096, 72)
    assert 4096 < kin.WARP_MAX_CELLS_PER_SM * torch.cuda.get_device_properties(0).multi_processor_count
    out = []
    for layout in (kin.LAYOUT_AUTO, WARP):
        Yd = dev(Y)
        kin.integrate(km, dev(T), dev(p), Yd, 1e-7, 1e-6, 1e-10, kin.RKCK, layout=layout)
        out.append(Yd.cpu().numpy())
    assert np.array_equal(out[0], out[1])


def test_warp_rkck_batch_equals_separate_and_nonfinite():
    name = "h2_9sp_rkck"
    m, km, om = mech(name)
    parts, singles = [], []
    for i, n in enumerate([50, 3, 400]):
        T, p, Y = states(name, m, n, 80 + i)
        if i == 2:
            Y[3, 7] = np.nan
        st = torch.zeros(n, dtype=torch.uint8, device=DEV)
        parts.append(kin.Cells(dev(T), dev(p), dev(Y), 1e-7, 1e-6, 1e-10, st))
        Ys = dev(Y)
        kin.integrate(km, dev(T), dev(p), Ys, 1e-7, 1e-6, 1e-10, kin.RKCK, layout=WARP)
        singles.append(Ys)
    kin.integrate_batch(km, parts, kin.RKCK, layout=WARP)
    torch.cuda.synchronize()
    for c, Ys in zip(parts, singles):
        assert torch.equal(torch.nan_to_num(c.Y), torch.nan_to_num(Ys))
    s2 = parts[2].status.cpu().numpy()
    assert s2[7] == kin.CELL_NONFINITE and (np.delete(s2, 7) == 0).all()
