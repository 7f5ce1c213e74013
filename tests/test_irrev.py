"""The reversible -> irreversible conversion of Appendix A (host tool), pinned
by the closed form of a balanced-heat-capacity reaction, the fit's exactness
at its three temperatures, and thermodynamic equilibrium of a converted pair
integrated by the oracle."""
import math

import numpy as np
import pytest

import oracle
from paper_1309_2710_gb300 import irrev, synth
from tests import mechs

R = 8.314462618


def test_balanced_heat_capacity_gives_the_exact_reverse_arrhenius_form():
    """With sum(nu cp) = 0, dH and dS are constant and
    k_f / K_c = A e^{-dS/R} (R T / p0')^{dn} T^beta e^{-(E - dH)/(R T)}:
    beta_r = beta + dn, E_r = E - dH, ln A_r = ln A - dS/R + dn ln(R / p0'),
    p0' = 101325 Pa in mol/cm^3 units (x 1e-6)."""
    cp = [29.0, 33.0, 40.0, 22.0]          # cp_A + cp_B = cp_C + cp_D
    Hf = [0.0, -50e3, -180e3, 30e3]
    S0 = [205.0, 188.0, 214.0, 115.0]
    lnA, beta, Ea = math.log(3e12), 0.4, 7.5e4
    for reac, prod in (([0, 1], [2, 3]), ([0, 1], [2])):
        nu = np.zeros(4)
        for s in prod:
            nu[s] += 1
        for s in reac:
            nu[s] -= 1
        if len(prod) == 1:                 # dn = -1: balance cp with the product alone
            cp2 = list(cp)
            cp2[2] = cp[0] + cp[1]
        else:
            cp2 = cp
        dH, dS, dn = nu @ Hf, nu @ S0, nu.sum()
        lnAr, br, Er = irrev.reverse_parameters(lnA, beta, Ea, cp2, Hf, S0, reac, prod)
        assert br == pytest.approx(beta + dn, abs=1e-9)
        assert Er == pytest.approx(Ea - dH, rel=1e-9, abs=1e-3)
        assert lnAr == pytest.approx(lnA - dS / R + dn * math.log(R / (101325.0 * 1e-6)), abs=1e-8)


def test_fit_is_exact_at_its_three_temperatures_and_close_between():
    m = synth.workload_mechanism("h2co_13sp_rkc_energy")
    S0 = synth.make_entropy(m, 5002)
    T3 = (300.0, 1000.0, 3000.0)
    worst = 0.0
    for j in range(m.n_reactions):
        lnAr, br, Er = irrev.reverse_parameters(m.lnA[j], m.beta[j], m.Ea[j], m.cp, m.Hf, S0,
                                                m.reac[j], m.prod[j], T3)
        for T in (300.0, 600.0, 1000.0, 1700.0, 3000.0):
            lnkf = m.lnA[j] + m.beta[j] * math.log(T) - m.Ea[j] / (R * T)
            exact = lnkf - math.log(irrev.equilibrium_constant(m.cp, m.Hf, S0, m.reac[j],
                                                               m.prod[j], T))
            fit = lnAr + br * math.log(T) - Er / (R * T)
            if T in T3:
                assert fit == pytest.approx(exact, abs=1e-8)
            worst = max(worst, abs(fit - exact))
    # constant-cp thermochemistry: the three-term form is close in between
    assert worst < 0.05, worst


def test_converted_pair_reaches_thermodynamic_equilibrium():
    """A <-> B (isomers, dn = 0) converted to two irreversible reactions and
    integrated by the oracle at fixed T far past the relaxation time:
    C_B / C_A -> K_c(T) at a fit temperature."""
    cp, Hf, S0 = [30.0, 36.0], [0.0, -8e3], [200.0, 190.0]
    m = mechs.mech([28.0, 28.0], [dict(reac=[0], prod=[1], A=2e6, beta=0.3, Ea=2e4)],
                   cp=cp, Hf=Hf, S0=S0)
    mi = irrev.to_irreversible(m, [True])
    assert len(mi.lnA) == 2 and list(mi.reac[1]) == [1, -1] and list(mi.prod[1]) == [0, -1]
    om = oracle.Mech(mi)
    T = 1000.0
    Kc = irrev.equilibrium_constant(cp, Hf, S0, [0], [1], T)
    kf = 2e6 * T ** 0.3 * math.exp(-2e4 / (R * T))
    Y = np.array([[0.9], [0.1]])
    Yn, st, _, _ = oracle.integrate(om, np.array([T]), np.array([101325.0]), Y,
                                    40.0 / (kf * (1 + 1 / Kc)), 1e-10, 1e-14, oracle.RKCK)
    assert st[0] == 0
    assert Yn[1, 0] / Yn[0, 0] == pytest.approx(Kc, rel=1e-7)


def test_third_body_and_falloff_reverses_keep_their_form():
    m = synth.workload_mechanism("ch4_53sp_rkc_mixed_energy")
    m.S0 = synth.make_entropy(m, 5003)
    rev = np.zeros(m.n_reactions, bool)
    rev[::3] = True
    mi = irrev.to_irreversible(m, rev)
    assert len(mi.lnA) == m.n_reactions + rev.sum()
    assert len(mi.eff) == np.count_nonzero(mi.rtype)
    q = 0
    for j in range(m.n_reactions):
        q += 1
        if rev[j]:
            assert mi.rtype[q] == m.rtype[j]
            assert list(mi.reac[q]) == list(m.prod[j]) and list(mi.prod[q]) == list(m.reac[j])
            q += 1


def test_converted_synthetic_mechanism_conserves_mass_and_elements():
    """The converted tables (27 reversible -> 54 irreversible reactions) keep
    every reaction balanced, and an oracle integration conserves mass."""
    m = synth.make_reversible_mechanism(13, 27, ("H", "O", "C", "N"), tb_frac=0.1, seed=1102)
    mi = irrev.to_irreversible(m, np.ones(27, bool))
    comp = np.asarray(m.comp)
    for j in range(len(mi.lnA)):
        a = sum(comp[s] for s in mi.reac[j] if s >= 0)
        b = sum(comp[s] for s in mi.prod[j] if s >= 0)
        assert np.array_equal(a, b)
    om = oracle.Mech(mi)
    T, p, Y = synth.make_states(mi, 16, T_range=(1800.0, 2800.0), seed=2102)
    Yn, st, _, _ = oracle.integrate(om, T, p, Y, 1e-4, 1e-8, 1e-14, oracle.RKC_POWER)
    assert (st == 0).all()
    assert np.abs(Yn.sum(0) - 1).max() < 1e-12
