"""GPU parity of the generated f (KIN_FEVAL_GENERATED): the mechanism's f as
straight-line code, compiled at run time into the lane-per-cell integrator,
against the FP64 oracle (both methods, both spectral-radius estimators,
ragged sizes, isothermal and with the energy equation), against the
table-driven kernels, through the automatic choice, the batched launch and a
CUDA graph; and the refusals outside its scope."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1309_2710_gb300 import synth  # noqa: E402
from tests.oracle_variants import reference  # noqa: E402
from tests.parity import compare, tol_rel_err  # noqa: E402

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1309_2710_gb300 import build as kbuild  # noqa: E402

kbuild.build()
from paper_1309_2710_gb300 import kin  # noqa: E402

DEV = torch.device("cuda:0")
GEN, TABLE, LANE = kin.FEVAL_GENERATED, kin.FEVAL_TABLE, kin.LAYOUT_LANE
_M = {}


def mech(name):
    if name not in _M:
        m = synth.workload_mechanism(name)
        _M[name] = (m, kin.Mechanism(m), oracle.Mech(m))
    return _M[name]


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device=DEV)


def run(km, T, p, Y, w, feval, sigma=None, layout=LANE, **kw):
    cells = T.shape[0]
    Yd = dev(Y)
    st = torch.full((cells,), 255, dtype=torch.uint8, device=DEV)
    sta = torch.zeros((cells, kin.NSTATS), dtype=torch.int32, device=DEV)
    kin.integrate(km, dev(T), dev(p), Yd, w["dt"], w["rtol"], w["atol"], w["method"], status=st, stats=sta,
                  sigma=w["sigma"] if sigma is None else sigma, layout=layout, feval=feval, **kw)
    torch.cuda.synchronize()
    return Yd.cpu().numpy(), st.cpu().numpy(), sta.cpu().numpy()


def omethod(method, sigma):
    if method == kin.RKCK:
        return oracle.RKCK
    return oracle.RKC_POWER if sigma == kin.SIGMA_POWER else oracle.RKC


@pytest.mark.parametrize("name,cells,sigma", [("h2co_13sp_rkc", 517, kin.SIGMA_GERSHGORIN),
                                              ("h2co_13sp_rkc", 300, kin.SIGMA_POWER),
                                              ("h2_9sp_rkck", 4096, None),
                                              ("h2_9sp_rkck", 33, None)])
def test_generated_against_oracle(name, cells, sigma):
    w = synth.WORKLOADS[name]
    m, km, om = mech(name)
    sigma = w["sigma"] if sigma is None else sigma
    T, p, Y = synth.workload_states(name, m, cells=cells, seed_offset=91)
    Yg, stg, stag = run(km, T, p, Y, w, GEN, sigma=sigma)
    Yo, sto, stao, fl = reference(m, T, p, Y, w["dt"], w["rtol"], w["atol"], omethod(w["method"], sigma))
    s = compare(Yg, Yo, stg, sto, stag, stao, w["atol"], w["rtol"], floor=fl)
    print("generated", name, cells, s)


@pytest.mark.parametrize("occupancy", [kin.OCC_DEFAULT, kin.OCC_HIGH])
def test_generated_against_tables(occupancy):
    """Same method and decisions as the table-driven kernel; f rounds its sums
    in another order, so the states agree within the tolerance scale."""
    name = "h2co_13sp_rkc"
    w = synth.WORKLOADS[name]
    m, km, om = mech(name)
    T, p, Y = synth.workload_states(name, m, cells=4000, seed_offset=92)
    a = run(km, T, p, Y, w, GEN, occupancy=occupancy)
    b = run(km, T, p, Y, w, TABLE, occupancy=occupancy)
    compare(a[0], b[0], a[1], b[1], a[2], b[2], w["atol"], w["rtol"])


def test_generated_launch_shapes_bit_identical():
    """The benchmark's candidate shapes (both register budgets, block sizes)
    give the same bits: each cell's arithmetic does not depend on which lane
    or launch shape integrates it."""
    name = "h2co_13sp_rkc"
    w = synth.WORKLOADS[name]
    m, km, om = mech(name)
    T, p, Y = synth.workload_states(name, m, cells=3000, seed_offset=96)
    ref = run(km, T, p, Y, w, GEN, block_threads=32, blocks_per_sm=16, occupancy=kin.OCC_DEFAULT)
    for bt, bps, occ in ((128, 4, kin.OCC_DEFAULT), (32, 20, kin.OCC_HIGH), (128, 6, kin.OCC_HIGH)):
        got = run(km, T, p, Y, w, GEN, block_threads=bt, blocks_per_sm=bps, occupancy=occ)
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[2], ref[2]), (bt, bps, occ)


def test_automatic_choice_uses_generated_for_large_calls():
    name = "h2co_13sp_rkc"
    w = synth.WORKLOADS[name]
    m, km, om = mech(name)
    cells = kin.GEN_MIN_CELLS
    T, p, Y = synth.workload_states(name, m, cells=cells, seed_offset=93)
    auto = run(km, T, p, Y, w, kin.FEVAL_AUTO)
    gen = run(km, T, p, Y, w, GEN)
    assert np.array_equal(auto[0], gen[0]) and np.array_equal(auto[2], gen[2])
    # and the tables below the threshold
    small = cells // 64
    auto_s = run(km, T[:small], p[:small], Y[:, :small], w, kin.FEVAL_AUTO)
    tab_s = run(km, T[:small], p[:small], Y[:, :small], w, TABLE)
    assert np.array_equal(auto_s[0], tab_s[0])
    idx = np.arange(0, cells, 97)
    Yo, sto, stao, _ = oracle.integrate(om, T[idx], p[idx], Y[:, idx], w["dt"], w["rtol"], w["atol"], oracle.RKC)
    e = tol_rel_err(gen[0][:, idx], Yo, w["atol"], w["rtol"])
    same = (gen[2][idx] == stao).all(axis=1)
    assert e[:, same].max() <= 1e-8 and same.mean() >= 0.99


def test_generated_batch_and_graph():
    name = "h2co_13sp_rkc"
    w = synth.WORKLOADS[name]
    m, km, om = mech(name)
    sizes = [700, 1, 1300]
    parts, alone = [], []
    for i, n in enumerate(sizes):
        T, p, Y = synth.workload_states(name, m, cells=n, seed_offset=94 + i)
        alone.append(run(km, T, p, Y, w, GEN))
        parts.append(kin.Cells(dev(T), dev(p), dev(Y), w["dt"], w["rtol"], w["atol"],
                               torch.zeros(n, dtype=torch.uint8, device=DEV),
                               torch.zeros((n, kin.NSTATS), dtype=torch.int32, device=DEV)))
    Y0 = [c.Y.clone() for c in parts]
    kin.integrate_batch(km, parts, kin.RKC, layout=LANE, feval=GEN, sigma=w["sigma"])
    torch.cuda.synchronize()
    for c, a in zip(parts, alone):
        assert np.array_equal(c.Y.cpu().numpy(), a[0]) and np.array_equal(c.stats.cpu().numpy(), a[2])
    # replayed from a CUDA graph (the first call above compiled and loaded f)
    ws = km.workspace(kin.RKC, kin.FP64, sum(sizes), layout=LANE, device=DEV, sigma=w["sigma"])
    stream = torch.cuda.Stream()
    for c, y0 in zip(parts, Y0):
        c.Y.copy_(y0)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        kin.integrate_batch(km, parts, kin.RKC, workspace=ws, layout=LANE, feval=GEN, sigma=w["sigma"])
    for c, y0 in zip(parts, Y0):
        c.Y.copy_(y0)
    g.replay()
    torch.cuda.synchronize()
    for c, a in zip(parts, alone):
        assert np.array_equal(c.Y.cpu().numpy(), a[0])


@pytest.mark.parametrize("name,cells", [("h2co_13sp_rkc_energy", 211), ("h2_9sp_rkck_energy", 333)])
def test_generated_energy_against_oracle(name, cells):
    """The energy equation with the generated f: T is a state component, k_j
    follows it inside f; against the FP64 oracle and the table-driven kernel."""
    w = synth.WORKLOADS[name]
    m, km, om = mech(name)
    T, p, Y = synth.workload_states(name, m, cells=cells, seed_offset=95)

    def go(feval):
        Td, Yd = dev(T), dev(Y)
        st = torch.full((cells,), 255, dtype=torch.uint8, device=DEV)
        sta = torch.zeros((cells, kin.NSTATS), dtype=torch.int32, device=DEV)
        kin.integrate(km, Td, dev(p), Yd, w["dt"], w["rtol"], w["atol"], w["method"], status=st, stats=sta,
                      sigma=w["sigma"], layout=LANE, energy=1, feval=feval)
        torch.cuda.synchronize()
        return np.vstack([Yd.cpu().numpy(), Td.cpu().numpy()]), st.cpu().numpy(), sta.cpu().numpy()

    g, t = go(GEN), go(TABLE)
    Yo, sto, stao, _, To = oracle.integrate(om, T, p, Y, w["dt"], w["rtol"], w["atol"],
                                            omethod(w["method"], w["sigma"]), energy=True)
    assert np.abs(To - T).max() > 1e-3
    frac = 0.05 if w["method"] == kin.RKC else 0.01
    compare(g[0], np.vstack([Yo, To]), g[1], sto, g[2], stao, w["atol"], w["rtol"], max_div_frac=frac)
    compare(g[0], t[0], g[1], t[1], g[2], t[2], w["atol"], w["rtol"], max_div_frac=frac)


@pytest.mark.parametrize("case", ["mixed", "warp", "large", "staging"])
def test_generated_refusals(case):
    name = {"large": "ch4_53sp_rkc_mixed"}.get(case, "h2co_13sp_rkc")
    m, km, om = mech(name)
    w = dict(synth.WORKLOADS[name])
    T, p, Y = synth.workload_states(name, m, cells=64)
    kw = dict(precision=kin.FP64)
    if case == "mixed":
        kw["precision"] = kin.MIXED
    if case == "staging":
        kw["staging"] = kin.STAGE_SHARED
    layout = kin.LAYOUT_WARP if case == "warp" else LANE
    with pytest.raises(kin.KinError) as e:
        run(km, T, p, Y, w, GEN, layout=layout, **kw)
    assert e.value.code == kin.KIN_EUNSUPPORTED
