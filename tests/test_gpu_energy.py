"""GPU parity of the constant-pressure energy equation (Eq. (E:energy)): T is
the (nS+1)-th state component, written back in place, and k_j, density and
concentrations follow it at every evaluation of f. Both layouts, both
methods, both precisions, against the FP64 oracle; plus the closed-form
adiabatic temperature rise and the host-buffer entry point."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1309_2710_gb300 import synth  # noqa: E402
from tests import mechs  # noqa: E402
from tests.oracle_variants import reference  # noqa: E402
from tests.parity import compare, compare_mixed, tol_rel_err  # noqa: E402

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1309_2710_gb300 import build as kbuild  # noqa: E402

kbuild.build()
from paper_1309_2710_gb300 import kin  # noqa: E402

DEV = torch.device("cuda:0")
_M = {}


def mech(name):
    if name not in _M:
        m = synth.workload_mechanism(name)
        _M[name] = (m, kin.Mechanism(m), oracle.Mech(m))
    return _M[name]


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device=DEV)


def run(km, T, p, Y, dt, method, precision=kin.FP64, sigma=kin.SIGMA_POWER, layout=kin.LAYOUT_AUTO,
        max_steps=20000, **shape):
    cells = T.shape[0]
    Td, Yd = dev(T), dev(Y)
    st = torch.full((cells,), 255, dtype=torch.uint8, device=DEV)
    sta = torch.zeros((cells, kin.NSTATS), dtype=torch.int32, device=DEV)
    kin.integrate(km, Td, dev(p), Yd, dt, 1e-6, 1e-10, method, precision, status=st, stats=sta,
                  max_steps=max_steps, sigma=sigma, layout=layout, energy=1, **shape)
    torch.cuda.synchronize()
    return Yd.cpu().numpy(), Td.cpu().numpy(), st.cpu().numpy(), sta.cpu().numpy()


def omethod(method, sigma):
    if method == kin.RKCK:
        return oracle.RKCK
    return oracle.RKC_POWER if sigma == kin.SIGMA_POWER else oracle.RKC


@pytest.mark.parametrize("name,cells,sigma,layout", [
    ("h2_9sp_rkck_energy", 333, None, kin.LAYOUT_LANE),
    ("h2co_13sp_rkc_energy", 517, kin.SIGMA_POWER, kin.LAYOUT_LANE),
    ("h2co_13sp_rkc_energy", 97, kin.SIGMA_GERSHGORIN, kin.LAYOUT_LANE),
    ("h2co_13sp_rkc_energy", 211, kin.SIGMA_POWER, kin.LAYOUT_WARP),
    ("ch4_53sp_rkc_mixed_energy", 65, kin.SIGMA_POWER, kin.LAYOUT_WARP),
    ("ch4_53sp_rkc_mixed_energy", 33, kin.SIGMA_POWER, kin.LAYOUT_LANE),
])
def test_energy_fp64_against_oracle(name, cells, sigma, layout):
    w = synth.WORKLOADS[name]
    m, km, om = mech(name)
    method = w["method"]
    sigma = w["sigma"] if sigma is None else sigma
    T, p, Y = synth.workload_states(name, m, cells=cells, seed_offset=61)
    Yg, Tg, stg, stag = run(km, T, p, Y, w["dt"], method, sigma=sigma, layout=layout)
    Yo, sto, stao, To, fl = reference(m, T, p, Y, w["dt"], w["rtol"], w["atol"],
                                      omethod(method, sigma), energy=True)
    assert np.abs(To - T).max() > 1e-3  # the temperature moved
    frac = 0.05 if sigma == kin.SIGMA_POWER and method == kin.RKC else 0.01
    s = compare(np.vstack([Yg, Tg]), np.vstack([Yo, To]), stg, sto, stag, stao, w["atol"], w["rtol"],
                max_div_frac=frac, floor=fl)
    print("energy", name, layout, s, "max |dT| %.2f K" % np.abs(To - T).max())


@pytest.mark.parametrize("layout", [kin.LAYOUT_WARP, kin.LAYOUT_LANE])
def test_energy_mixed_against_fp64_oracle(layout):
    """FP32 rates (the exponents formed in FP64), FP64 state including T, FP64
    spectral-radius evaluations: within 1e-5 of the FP64 oracle per component."""
    name = "ch4_53sp_rkc_mixed_energy"
    w = synth.WORKLOADS[name]
    m, km, om = mech(name)
    T, p, Y = synth.workload_states(name, m, cells=256, seed_offset=62)
    Yg, Tg, stg, stag = run(km, T, p, Y, w["dt"], kin.RKC, kin.MIXED, layout=layout)
    idx = np.arange(0, 256, 4)
    Yo, sto, stao, _, To = oracle.integrate(om, T[idx], p[idx], Y[:, idx], w["dt"], w["rtol"],
                                            w["atol"], oracle.RKC_POWER, energy=True)
    e = tol_rel_err(np.vstack([Yg[:, idx], Tg[idx]]), np.vstack([Yo, To]), w["atol"], w["rtol"])
    print("energy mixed", layout, "T %.3e" % e[-1].max(),
          compare_mixed(np.vstack([Yg[:, idx], Tg[idx]]), np.vstack([Yo, To]), stg[idx], sto, stag[idx], stao,
                        w["atol"], w["rtol"]))


def test_energy_layouts_agree():
    name = "h2co_13sp_rkc_energy"
    m, km, om = mech(name)
    T, p, Y = synth.workload_states(name, m, cells=400, seed_offset=63)
    a = run(km, T, p, Y, 1e-6, kin.RKC, layout=kin.LAYOUT_LANE)
    b = run(km, T, p, Y, 1e-6, kin.RKC, layout=kin.LAYOUT_WARP)
    compare(np.vstack([a[0], a[1]]), np.vstack([b[0], b[1]]), a[2], b[2], a[3], b[3], 1e-10, 1e-6,
            max_div_frac=0.05)


@pytest.mark.parametrize("method,layout", [(kin.RKCK, kin.LAYOUT_LANE), (kin.RKC, kin.LAYOUT_LANE),
                                           (kin.RKC, kin.LAYOUT_WARP)])
def test_energy_adiabatic_rise_closed_form(method, layout):
    """A -> B with T-independent k, equal W and cp: T(t) = T0 + dH (Y_A0 -
    Y_A(t)) / cp with Y_A(t) = Y_A0 exp(-k t) (enthalpy conservation)."""
    k, dH, cp = 1e6, 1e5, 30.0
    m = mechs.mech([28.0, 28.0, 28.0], [dict(reac=[0], prod=[1], A=k)], cp=[cp] * 3,
                   Hf=[0.0, -dH, 0.0])
    km = kin.Mechanism(m)
    cells = 40
    T = np.full(cells, 1000.0)
    p = np.full(cells, 101325.0)
    Y = np.zeros((3, cells))
    Y[0] = np.linspace(0.02, 0.2, cells)
    Y[2] = 1.0 - Y[0]
    Td, Yd = dev(T), dev(Y)
    st = torch.zeros(cells, dtype=torch.uint8, device=DEV)
    kin.integrate(km, Td, dev(p), Yd, 1e-6, 1e-10, 1e-14, method, status=st, energy=1,
                  layout=layout, sigma=kin.SIGMA_POWER)
    torch.cuda.synchronize()
    assert int(st.max()) == 0
    ya = Y[0] * math.exp(-k * 1e-6)
    rise = dH * (Y[0] - ya) / cp
    np.testing.assert_allclose(Yd.cpu().numpy()[0], ya, rtol=1e-7)
    np.testing.assert_allclose(Td.cpu().numpy() - T, rise, rtol=1e-7)


def test_energy_host_buffers_write_T_back():
    name = "h2co_13sp_rkc_energy"
    m, km, om = mech(name)
    T, p, Y = synth.workload_states(name, m, cells=300, seed_offset=64)
    Yd_, Td_, _, _ = run(km, T, p, Y, 1e-6, kin.RKC)
    Th = torch.as_tensor(T.copy()).pin_memory()
    Yh = torch.as_tensor(np.ascontiguousarray(Y)).pin_memory()
    kin.integrate_host(km, Th, torch.as_tensor(p).pin_memory(), Yh, 1e-6, 1e-6, 1e-10, kin.RKC,
                       sigma=kin.SIGMA_POWER, energy=1)
    torch.cuda.synchronize()
    assert np.array_equal(Th.numpy(), Td_) and np.array_equal(Yh.numpy(), Yd_)


def test_energy_needs_thermochemistry():
    m = synth.workload_mechanism("h2co_13sp_rkc")  # no cp / Hf
    km = kin.Mechanism(m)
    T, p, Y = synth.workload_states("h2co_13sp_rkc", m, cells=4)
    with pytest.raises(kin.KinError) as e:
        kin.integrate(km, dev(T), dev(p), dev(Y), 1e-6, 1e-6, 1e-10, kin.RKC, energy=1)
    assert e.value.code == kin.KIN_EUNSUPPORTED


def test_energy_off_leaves_T_untouched():
    name = "h2co_13sp_rkc_energy"
    m, km, om = mech(name)
    T, p, Y = synth.workload_states(name, m, cells=64, seed_offset=65)
    Td = dev(T)
    kin.integrate(km, Td, dev(p), dev(Y), 1e-6, 1e-6, 1e-10, kin.RKC)
    torch.cuda.synchronize()
    assert np.array_equal(Td.cpu().numpy(), T)
