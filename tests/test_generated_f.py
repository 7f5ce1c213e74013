"""The generated f (kin_generated_f_source) on the CPU: the library writes the
mechanism-specific source, g++ compiles it behind a small shim of the device
types, and every evaluation is compared with the oracle's f (Eqs. (E:mass),
(E:spec-rate), (E:rxn-rate)) for the same state and rate constants, and with
the energy equation (Eq. (E:energy)) for mechanisms with thermochemistry.
Runs without a GPU; the GPU tests run the same source inside the integrator."""
import ctypes
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_1309_2710_gb300 import kin, synth
from tests import mechs

SHIM = r"""
#include <cmath>
#define __device__
#define __forceinline__ inline
namespace kin {
struct MechDev {};
template <typename T> struct Lane {
    T* p;
    int s;
    T& operator[](int i) const { return p[(long)i * s]; }
};
template <typename R> struct Tab;
template <> struct Tab<double> { static double inv(double a) { return 1.0 / a; } };
inline double ddiv(double a, double b) { return a / b; }
constexpr double R_GAS = 8.314462618, T_REF = 298.15;
using std::exp;
using std::fma;
using std::log;
}
#include "gen_f.inc"
extern "C" void gen_f(double Ctot, double* K, double* KR, double* x, double* out)
{
    kin::Lane<double> k{K, 1}, kr{KR, 1}, xx{x, 1}, o{out, 1}, none{nullptr, 1};
    kin::GenF::eval<double, double>(kin::MechDev{}, Ctot, 1.0 / Ctot, k, kr, none, none, xx, o);
}
#ifdef GEN_ENERGY
extern "C" void gen_f_energy(double p, double* x, double* out)
{
    kin::Lane<double> xx{x, 1}, o{out, 1}, none{nullptr, 1};
    kin::GenF::eval_energy<double>(kin::MechDev{}, p, none, none, xx, o);
}
#endif
"""

R_GAS = 8.314462618


def compile_generated(m, tmp_path):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    src = kin.generated_f_source(m)
    (tmp_path / "gen_f.inc").write_text(src)
    (tmp_path / "shim.cpp").write_text(SHIM)
    so = str(tmp_path / "gen_f.so")
    energy = "eval_energy" in src
    subprocess.run(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", "-o", so, str(tmp_path / "shim.cpp")]
                   + (["-DGEN_ENERGY"] if energy else []), check=True, capture_output=True, cwd=tmp_path)
    L = ctypes.CDLL(so)
    L.gen_f.argtypes = [ctypes.c_double] + [ctypes.c_void_p] * 4
    if energy:
        L.gen_f_energy.argtypes = [ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]
    return L, src


def generated_rates(L, om, m, T, p, y):
    k, k0 = oracle.rate_constants(om, T)
    fo = np.flatnonzero(np.asarray(m.rtype) == 2)
    kr = np.ascontiguousarray(k0[fo] / k[fo]) if fo.size else np.zeros(1)
    k = np.ascontiguousarray(k)
    x = np.ascontiguousarray(y, dtype=np.float64)
    out = np.empty(len(m.W))
    ptr = lambda a: a.ctypes.data
    L.gen_f(p * 1e-6 / (R_GAS * T), ptr(k), ptr(kr), ptr(x), ptr(out))
    return out


@pytest.mark.parametrize("name", ["h2_9sp_rkck", "h2co_13sp_rkc"])
def test_generated_f_equals_the_oracle(name, tmp_path):
    m = synth.workload_mechanism(name)
    om = oracle.Mech(m)
    L, src = compile_generated(m, tmp_path)
    T, p, Y = synth.workload_states(name, m, cells=64, seed_offset=81)
    for c in range(64):
        ref = oracle.rates(om, T[c], p[c], Y[:, c])
        got = generated_rates(L, om, m, T[c], p[c], Y[:, c])
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max(), c
    # one accumulation per net stoichiometric nonzero, one block per reaction
    nnz = sum(int(np.sum(m.prod[j] == i) != np.sum(m.reac[j] == i))
              for j in range(len(m.lnA)) for i in range(len(m.W)))
    assert src.count("fma(") == nnz
    assert src.count("// reaction ") == len(m.lnA)


def test_generated_f_third_body_falloff_and_inert(tmp_path):
    """Every reaction form: A + A -> B (second order in one species), third
    body with an efficiency of exactly 1 and of 0, Lindemann falloff, a
    reaction whose product equals a reactant, and an inert species."""
    W = [2.016, 31.998, 18.015, 28.014]
    rx = [dict(reac=[0, 0], prod=[2], A=3e9, beta=0.5, Ea=4e4),
          dict(reac=[0, 1], prod=[2, 2], A=1e8, type=1),
          dict(reac=[2], prod=[0, 1], A=2e12, beta=-0.3, Ea=1.2e5, type=2, A0=5e15, Ea0=9e4),
          dict(reac=[1, 2], prod=[1, 0], A=4e10, Ea=7e4)]
    eff = [[1.0, 0.0, 2.5, 0.7], [1.3, 1.0, 0.0, 2.0]]
    m = mechs.mech(W, rx, eff_rows=eff)
    om = oracle.Mech(m)
    L, src = compile_generated(m, tmp_path)
    assert "out[3] = 0.0;" in src  # the inert species
    rng = np.random.default_rng(3)
    for _ in range(40):
        y = rng.uniform(0.01, 1.0, 4)
        y /= y.sum()
        T, p = rng.uniform(900, 2500), rng.uniform(5e4, 2e6)
        ref = oracle.rates(om, T, p, y)
        got = generated_rates(L, om, m, T, p, y)
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("name", ["h2co_13sp_rkc_energy", "h2_9sp_rkck_energy"])
def test_generated_energy_f_equals_the_oracle(name, tmp_path):
    """The form with the energy equation: k_j from the state's T inside f, and
    dT/dt = -(sum_i H_i omega_i) / (rho cp) as the last component."""
    m = synth.workload_mechanism(name)
    om = oracle.Mech(m)
    L, src = compile_generated(m, tmp_path)
    assert "eval_energy" in src
    T, p, Y = synth.workload_states(name, m, cells=48, seed_offset=82)
    nS = len(m.W)
    for c in range(48):
        y = np.ascontiguousarray(np.append(Y[:, c], T[c]))
        ref = oracle.rates_energy(om, p[c], y)
        out = np.empty(nS + 1)
        L.gen_f_energy(float(p[c]), y.ctypes.data, out.ctypes.data)
        assert np.abs(out[:nS] - ref[:nS]).max() <= 1e-12 * np.abs(ref[:nS]).max(), c
        assert abs(out[nS] - ref[nS]) <= 1e-12 * abs(ref[nS]), c
        # and the isothermal form at this T is the same species rows
        iso = generated_rates(L, om, m, T[c], p[c], Y[:, c])
        assert np.abs(iso - out[:nS]).max() <= 1e-12 * np.abs(ref[:nS]).max()


def test_generated_energy_f_falloff(tmp_path):
    W = [2.016, 31.998, 18.015, 28.014]
    rx = [dict(reac=[0, 0], prod=[2], A=3e9, beta=0.5, Ea=4e4),
          dict(reac=[2], prod=[0, 1], A=2e12, beta=-0.3, Ea=1.2e5, type=2, A0=5e15, beta0=0.2, Ea0=9e4),
          dict(reac=[0, 1], prod=[2, 2], A=1e8, type=1)]
    m = mechs.mech(W, rx, eff_rows=[[1.0, 0.5, 2.5, 0.7], [1.3, 1.0, 0.0, 2.0]],
                   cp=[29.0, 29.5, 33.6, 29.1], Hf=[0.0, 0.0, -2.418e5, 0.0])
    om = oracle.Mech(m)
    L, src = compile_generated(m, tmp_path)
    rng = np.random.default_rng(4)
    for _ in range(30):
        y = rng.uniform(0.01, 1.0, 4)
        y /= y.sum()
        y = np.append(y, rng.uniform(900, 2500))
        p = rng.uniform(5e4, 2e6)
        ref = oracle.rates_energy(om, p, y)
        out = np.empty(5)
        L.gen_f_energy(p, y.ctypes.data, out.ctypes.data)
        assert np.abs(out - ref).max() <= 1e-12 * np.abs(ref).max()


def test_generated_f_scope():
    big = synth.workload_mechanism("ch4_53sp_rkc_mixed")
    with pytest.raises(kin.KinError) as e:
        kin.generated_f_source(big)
    assert e.value.code == kin.KIN_EUNSUPPORTED
    bad = mechs.mech([1.0, 2.0], [dict(reac=[0], prod=[5], A=1.0)])
    with pytest.raises(kin.KinError) as e:
        kin.generated_f_source(bad)
    assert e.value.code == kin.KIN_EINVAL


def test_generated_f_degenerate_mechanisms(tmp_path):
    """No reactions, and a single species: f is identically zero, and the
    source still compiles (the mixture sums have one or no odd terms)."""
    for W, rx in (([28.0], []), ([2.0, 32.0, 18.0], [])):
        m = mechs.mech(W, rx)
        om = oracle.Mech(m)
        sub = tmp_path / ("n%d" % len(W))
        sub.mkdir()
        L, src = compile_generated(m, sub)
        assert "fma(" not in src
        y = np.full(len(W), 1.0 / len(W))
        got = generated_rates(L, om, m, 1500.0, 101325.0, y)
        assert np.array_equal(got, np.zeros(len(W)))
        assert np.array_equal(oracle.rates(om, 1500.0, 101325.0, y), np.zeros(len(W)))
