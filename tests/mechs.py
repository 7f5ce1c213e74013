"""Hand-built tiny mechanisms for the oracle pins (plain arrays)."""
import types

import numpy as np


def mech(W, reactions, eff_rows=None, cp=None, Hf=None, S0=None):
    """reactions: list of dicts with reac, prod (species index lists of length
    <= 2), A, beta, Ea, type (0/1/2), and for falloff A0, beta0, Ea0. cp, Hf:
    optional species thermochemistry (J/(mol K), J/mol) for the energy
    equation."""
    nR = len(reactions)
    reac = np.full((nR, 2), -1, np.int32)
    prod = np.full((nR, 2), -1, np.int32)
    lnA = np.zeros(nR); beta = np.zeros(nR); Ea = np.zeros(nR)
    lnA0 = np.zeros(nR); beta0 = np.zeros(nR); Ea0 = np.zeros(nR)
    rtype = np.zeros(nR, np.int8)
    for j, r in enumerate(reactions):
        reac[j, :len(r["reac"])] = r["reac"]
        prod[j, :len(r["prod"])] = r["prod"]
        lnA[j] = np.log(r["A"]); beta[j] = r.get("beta", 0.0); Ea[j] = r.get("Ea", 0.0)
        rtype[j] = r.get("type", 0)
        if rtype[j] == 2:
            lnA0[j] = np.log(r["A0"]); beta0[j] = r.get("beta0", 0.0); Ea0[j] = r.get("Ea0", 0.0)
    nM = int(np.count_nonzero(rtype))
    eff = np.zeros((nM, len(W))) if eff_rows is None else np.asarray(eff_rows, float)
    return types.SimpleNamespace(W=np.asarray(W, float), lnA=lnA, beta=beta, Ea=Ea,
                                 reac=reac, prod=prod, rtype=rtype, eff=eff,
                                 lnA0=lnA0, beta0=beta0, Ea0=Ea0,
                                 cp=None if cp is None else np.asarray(cp, float),
                                 Hf=None if Hf is None else np.asarray(Hf, float),
                                 S0=None if S0 is None else np.asarray(S0, float))


def a_to_b(k, W=28.0):
    """A -> B, unimolecular, equal molar masses: dY_A/dt = -k Y_A exactly."""
    return mech([W, W], [dict(reac=[0], prod=[1], A=k)])


def chain(ks, W=20.0):
    """A_0 -> A_1 -> ... -> A_n, unimolecular with rates ks."""
    n = len(ks) + 1
    return mech([W] * n, [dict(reac=[i], prod=[i + 1], A=k) for i, k in enumerate(ks)])
