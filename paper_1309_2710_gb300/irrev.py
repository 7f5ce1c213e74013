"""Reversible -> irreversible reaction conversion (the paper's Appendix A).

The kernels integrate irreversible reactions only: a reversible reaction
would need its equilibrium constant, and with it the species' Gibbs
functions, inside every evaluation of f. Instead each reversible reaction is
split once, on the host, into its forward reaction and a reverse reaction
whose Arrhenius parameters (A_r, beta_r, E_r) are fitted so that
k_r(T) = k_f(T) / K_c(T) holds exactly at three temperatures T1 < T2 < T3
(Appendix A; the paper follows Turanyi's procedure):

    ln k_r(T_i) = ln A_r + beta_r ln T_i - (E_r / R) / T_i ,   i = 1, 2, 3,

a linear system in (ln A_r, beta_r, E_r / R), solved here directly.

The equilibrium constant in concentration units (mol/cm^3) is
K_c = K_p (p0 / (R T))^dn with dn = sum(products) - sum(reactants),
K_p = exp(-dG0 / (R T)), dG0 = sum_i nu_i (H_i(T) - T S_i(T)), and with the
constant heat capacities of the synthetic thermochemistry
H_i(T) = Hf_i + cp_i (T - 298.15), S_i(T) = S0_i + cp_i ln(T / 298.15) at
p0 = 1 atm. When the reaction's dcp = 0, k_f / K_c is exactly of Arrhenius
form and the fit reproduces it at every temperature; otherwise it is exact
at T1, T2, T3 and close in between.

Host-side preprocessing (numpy), not part of the integration hot path.
"""
from __future__ import annotations

import copy
from typing import Sequence, Tuple

import numpy as np

R_GAS = 8.314462618  # J/(mol K)
P0 = 101325.0  # Pa, standard state of S0
T_REF = 298.15  # K


def _stoich(reac: Sequence[int], prod: Sequence[int], n_species: int) -> np.ndarray:
    nu = np.zeros(n_species)
    for s in prod:
        if s >= 0:
            nu[s] += 1.0
    for s in reac:
        if s >= 0:
            nu[s] -= 1.0
    return nu


def equilibrium_constant(cp, Hf, S0, reac, prod, T) -> np.ndarray:
    """K_c(T) of reac -> prod in (mol/cm^3)^dn, for T scalar or array."""
    T = np.asarray(T, dtype=np.float64)
    cp, Hf, S0 = (np.asarray(a, dtype=np.float64) for a in (cp, Hf, S0))
    nu = _stoich(reac, prod, len(cp))
    dH = nu @ Hf + (nu @ cp) * (T - T_REF)
    dS = nu @ S0 + (nu @ cp) * np.log(T / T_REF)
    dn = nu.sum()
    lnKp = -(dH - T * dS) / (R_GAS * T)
    return np.exp(lnKp + dn * np.log(P0 * 1e-6 / (R_GAS * T)))


def fit_arrhenius(T3: Sequence[float], lnk: Sequence[float]) -> Tuple[float, float, float]:
    """(ln A, beta, E [J/mol]) with ln k = ln A + beta ln T - E / (R T) at the
    three temperatures."""
    T3 = np.asarray(T3, dtype=np.float64)
    M = np.column_stack([np.ones(3), np.log(T3), -1.0 / T3])
    lnA, beta, TaR = np.linalg.solve(M, np.asarray(lnk, dtype=np.float64))
    return float(lnA), float(beta), float(TaR * R_GAS)


def reverse_parameters(lnA, beta, Ea, cp, Hf, S0, reac, prod,
                       temperatures=(300.0, 1000.0, 3000.0)) -> Tuple[float, float, float]:
    """Fitted reverse Arrhenius parameters (ln A_r, beta_r, E_r [J/mol]) of one
    reaction with forward parameters (ln A, beta, E [J/mol])."""
    T3 = np.asarray(temperatures, dtype=np.float64)
    lnkf = lnA + beta * np.log(T3) - Ea / (R_GAS * T3)
    lnkr = lnkf - np.log(equilibrium_constant(cp, Hf, S0, reac, prod, T3))
    return fit_arrhenius(T3, lnkr)


def to_irreversible(mech, reversible: Sequence[bool], temperatures=(300.0, 1000.0, 3000.0)):
    """A copy of `mech` (mechanism arrays W, lnA, beta, Ea, reac, prod, rtype,
    eff, lnA0, beta0, Ea0 with the thermochemistry cp, Hf, S0, e.g. a
    synth.Mechanism) in which every reaction flagged reversible is followed
    by its fitted reverse reaction.
    A third-body reaction's reverse keeps its efficiencies. A falloff
    reaction's reverse fits both limits with the same K_c (k0_r = k0 / K_c),
    so Pr and the blending are those of the forward reaction."""
    if mech.cp is None or mech.Hf is None or getattr(mech, "S0", None) is None:
        raise ValueError("the conversion needs cp, Hf and S0")
    n_reactions, n_species = len(mech.lnA), len(mech.W)
    rev = np.asarray(reversible, dtype=bool)
    if rev.shape != (n_reactions,):
        raise ValueError("one flag per reaction")
    rows = []        # new reactions in order: (source j, is_reverse)
    for j in range(n_reactions):
        rows.append((j, False))
        if rev[j]:
            rows.append((j, True))
    nR = len(rows)
    reac = np.full((nR, 2), -1, np.int32)
    prod = np.full((nR, 2), -1, np.int32)
    lnA, beta, Ea = np.zeros(nR), np.zeros(nR), np.zeros(nR)
    lnA0, beta0, Ea0 = np.zeros(nR), np.zeros(nR), np.zeros(nR)
    rtype = np.zeros(nR, np.int8)
    eff_rows = []
    src_row = np.cumsum(np.asarray(mech.rtype) != 0) - 1  # efficiency row of each source reaction
    for q, (j, is_rev) in enumerate(rows):
        rtype[q] = mech.rtype[j]
        if mech.rtype[j] != 0:
            eff_rows.append(np.asarray(mech.eff)[src_row[j]])
        if not is_rev:
            reac[q], prod[q] = mech.reac[j], mech.prod[j]
            lnA[q], beta[q], Ea[q] = mech.lnA[j], mech.beta[j], mech.Ea[j]
            lnA0[q], beta0[q], Ea0[q] = mech.lnA0[j], mech.beta0[j], mech.Ea0[j]
            continue
        reac[q], prod[q] = mech.prod[j], mech.reac[j]
        lnA[q], beta[q], Ea[q] = reverse_parameters(mech.lnA[j], mech.beta[j], mech.Ea[j], mech.cp,
                                                    mech.Hf, mech.S0, mech.reac[j], mech.prod[j],
                                                    temperatures)
        if mech.rtype[j] == 2:
            lnA0[q], beta0[q], Ea0[q] = reverse_parameters(mech.lnA0[j], mech.beta0[j], mech.Ea0[j],
                                                           mech.cp, mech.Hf, mech.S0, mech.reac[j],
                                                           mech.prod[j], temperatures)
    out = copy.copy(mech)
    for k, v in dict(lnA=lnA, beta=beta, Ea=Ea, reac=reac, prod=prod, rtype=rtype,
                     eff=np.asarray(eff_rows).reshape(len(eff_rows), n_species),
                     lnA0=lnA0, beta0=beta0, Ea0=Ea0).items():
        setattr(out, k, v)
    return out
