"""Seeded synthetic mechanisms and initial states.

This module only synthesises inputs. It contains no rate, integrator, norm or
step-control arithmetic. The integrator and the oracle both take its output as
plain arrays.

The paper measures on four published mechanisms (9/38, 13/54, 53/634 and
111/1566 species/irreversible reactions; Sections 3.1-3.4). Those mechanism
files are not available here, so each one is replaced by a seeded synthetic
mechanism with the same species and reaction counts:

* Species are small atom vectors over the mechanism's elements (at most
  2 C, 4 H, 3 O, 2 N). An oxidiser {O:2}, a fuel ({H:2}, or {C:1,H:4} when
  carbon is present) and an inert diluent {N:2} are always included. The
  diluent never reacts.
* Every reaction is a two-to-two pair exchange ``a + b -> c + d`` with
  ``atoms(a) + atoms(b) == atoms(c) + atoms(d)``, so atoms and mass balance by
  construction. Both the forward and products are drawn at random.
* Arrhenius parameters: A log-uniform in [1e8, 1e14] (cm-mol-s units),
  beta uniform in [-1, 1], Ea uniform in [0, 2e5] J/mol; the 111-species
  mechanism of the batched workload draws A in [10^11.5, 10^17.5] and Ea in
  [1e5, 3e5] J/mol (see WORKLOADS).
* Third-body and Lindemann falloff reactions get a dense efficiency row
  drawn uniformly from [0.5, 3] over all species. The low-pressure limit of a
  falloff reaction has log10(A0/A) ~ U(3, 7), beta0 = beta and Ea0 = 0.8 Ea.

Initial states mix fuel and oxidiser at an equivalence ratio drawn from
U(0.5, 2), add 3.76 mol of diluent per mol of oxidiser, spread 1 % of the mass
over all reactive species and apply 1 % multiplicative noise. The paper
samples its states from ignition runs instead (Section 3); those runs need the
real mechanisms.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

ATOMIC_MASS = {"H": 1.008, "C": 12.011, "N": 14.007, "O": 15.999}
MAX_ATOMS = {"C": 2, "H": 4, "O": 3, "N": 2}
ATM = 101325.0

PLAIN, THIRD_BODY, FALLOFF = 0, 1, 2


@dataclasses.dataclass
class Mechanism:
    """Mechanism tables in the layout the C ABI takes (all host numpy arrays).

    ``reac``/``prod`` are ``[n_reactions, 2]`` species indices, -1 for an empty
    slot. ``eff`` has one row per non-plain reaction, in reaction order.
    ``lnA0``/``beta0``/``Ea0`` are only read for falloff reactions.
    """

    names: List[str]
    elements: List[str]
    comp: np.ndarray  # [n_species, n_elements] atom counts
    W: np.ndarray  # [n_species] g/mol
    lnA: np.ndarray  # [n_reactions]
    beta: np.ndarray
    Ea: np.ndarray  # J/mol
    reac: np.ndarray  # int32 [n_reactions, 2]
    prod: np.ndarray  # int32 [n_reactions, 2]
    rtype: np.ndarray  # int8 [n_reactions]
    eff: np.ndarray  # [n_M, n_species]
    lnA0: np.ndarray
    beta0: np.ndarray
    Ea0: np.ndarray
    fuel: int
    oxidiser: int
    diluent: int  # -1 when the element set has no N
    seed: int
    cp: Optional[np.ndarray] = None  # [n_species] J/(mol K), for the energy equation
    Hf: Optional[np.ndarray] = None  # [n_species] J/mol at 298.15 K
    S0: Optional[np.ndarray] = None  # [n_species] J/(mol K) at 298.15 K and 1 atm (equilibrium
    #                                  constants of reversible reactions)

    @property
    def n_species(self) -> int:
        return int(self.W.shape[0])

    @property
    def n_reactions(self) -> int:
        return int(self.lnA.shape[0])

    @property
    def n_third_body_rows(self) -> int:
        return int(self.eff.shape[0])


def _name(vec: Tuple[int, ...], elements: Sequence[str]) -> str:
    order = [e for e in ("C", "H", "O", "N") if e in elements]
    out = ""
    for e in order:
        n = vec[elements.index(e)]
        if n:
            out += e + (str(n) if n > 1 else "")
    return out


def _vec(d: Dict[str, int], elements: Sequence[str]) -> Tuple[int, ...]:
    return tuple(int(d.get(e, 0)) for e in elements)


def _add(a, b):
    return tuple(x + y for x, y in zip(a, b))


def _pair_exchanges(species: List[Tuple[int, ...]]):
    """Map atom sum -> list of unordered index pairs (i <= j) with that sum."""
    table: Dict[Tuple[int, ...], List[Tuple[int, int]]] = {}
    for i in range(len(species)):
        for j in range(i, len(species)):
            table.setdefault(_add(species[i], species[j]), []).append((i, j))
    return table


def _grow_pool(reactive, cands, diluent_vec, target, rng, sample=24) -> None:
    """Add species to ``reactive`` until it holds ``target`` entries.

    A candidate ``c`` can join when ``c + d`` equals the atom sum of a pool
    pair for some partner ``d`` (already pooled, or joining with it). Among a
    random sample of joinable candidates the one with the most such pairs is
    taken, which keeps the number of distinct balanced reactions high.
    """
    in_cands = set(cands)
    while len(reactive) < target:
        sums = list(_pair_exchanges(reactive))
        pool = set(reactive)
        best = None
        for idx in rng.permutation(len(cands)):
            c = cands[idx]
            if c in pool:
                continue
            partners = []
            for s_vec in sums:
                d = tuple(x - y for x, y in zip(s_vec, c))
                if min(d) < 0 or sum(d) == 0 or d == diluent_vec:
                    continue
                if d in pool or d in in_cands:
                    partners.append(d)
            pooled = [d for d in partners if d in pool or d == c]
            if not pooled and (not partners or len(reactive) + 2 > target):
                continue
            if len(reactive) < 40:
                # exact: ordered pair exchanges the enlarged pool offers
                extra = [c] if pooled else [c, partners[0]]
                score = sum(len(v) * (len(v) - 1)
                            for v in _pair_exchanges(reactive + extra).values())
            else:
                score = 2 * len(pooled) + len(partners)
            if best is None or score > best[0]:
                best = (score, c, pooled, partners)
            sample -= 1
            if sample <= 0:
                break
        if best is None:
            raise ValueError("element set too small for %d species" % (target + 1))
        _, c, pooled, partners = best
        reactive.append(c)
        if not pooled:
            reactive.append(partners[int(rng.integers(0, len(partners)))])
        sample = 24


def make_mechanism(n_species: int, n_reactions: int, elements: Sequence[str],
                   tb_frac: float = 0.0, fo_frac: float = 0.0,
                   seed: int = 0, log10_A: Tuple[float, float] = (8.0, 14.0),
                   Ea_range: Tuple[float, float] = (0.0, 2.0e5)) -> Mechanism:
    """Draw a balanced, irreversible synthetic mechanism (see module doc).
    log10_A and Ea_range bound the log-uniform pre-exponential factors
    (cm-mol-s) and the uniform activation energies (J/mol); the draws behind
    them do not depend on the bounds."""
    elements = list(elements)
    rng = np.random.default_rng(seed)
    has_n = "N" in elements
    diluent_vec = _vec({"N": 2}, elements) if has_n else None
    ox_vec = _vec({"O": 2}, elements)
    fuel_vec = _vec({"C": 1, "H": 4} if "C" in elements else {"H": 2}, elements)

    ranges = [range(MAX_ATOMS[e] + 1) for e in elements]
    cands = []
    for v in np.ndindex(*[len(r) for r in ranges]):
        t = tuple(int(x) for x in v)
        if sum(t) == 0 or t in (diluent_vec, ox_vec, fuel_vec):
            continue
        cands.append(t)
    # When the N-free candidates cannot fill the pool, a reactive nitrogen
    # carrier {N:1,O:1} seeds N chemistry (N species cannot appear otherwise).
    no_vec = _vec({"N": 1, "O": 1}, elements) if has_n else None
    n_no_n = sum(1 for t in cands if not has_n or t[elements.index("N")] == 0)
    reactive = [ox_vec, fuel_vec]
    if has_n and n_no_n + 2 < n_species - 1:
        reactive.append(no_vec)
    n_reactive_target = n_species - (1 if has_n else 0)

    _grow_pool(reactive, cands, diluent_vec, n_reactive_target, rng)

    species = list(reactive) + ([diluent_vec] if has_n else [])
    comp = np.array(species, dtype=np.int32)
    masses = np.array([ATOMIC_MASS[e] for e in elements])
    W = comp @ masses
    names = [_name(v, elements) for v in species]

    tab = _pair_exchanges(list(reactive))
    nreact = len(reactive)
    reac = np.full((n_reactions, 2), -1, dtype=np.int32)
    prod = np.full((n_reactions, 2), -1, dtype=np.int32)
    seen = set()
    for j in range(n_reactions):
        for attempt in range(10000):
            a, b = sorted(int(x) for x in rng.integers(0, nreact, size=2))
            opts = [p for p in tab[_add(reactive[a], reactive[b])] if p != (a, b)]
            if not opts:
                continue
            c, d = opts[int(rng.integers(0, len(opts)))]
            key = (a, b, c, d)
            if key in seen and attempt < 5000:
                continue
            seen.add(key)
            reac[j] = (a, b)
            prod[j] = (c, d)
            break
        else:  # pragma: no cover - the species pool always has exchanges
            raise RuntimeError("could not draw a balanced reaction")

    lnA = np.log(10.0) * rng.uniform(log10_A[0], log10_A[1], n_reactions)
    beta = rng.uniform(-1.0, 1.0, n_reactions)
    Ea = rng.uniform(Ea_range[0], Ea_range[1], n_reactions)

    rtype = np.zeros(n_reactions, dtype=np.int8)
    n_tb = int(round(tb_frac * n_reactions))
    n_fo = int(round(fo_frac * n_reactions))
    perm = rng.permutation(n_reactions)
    rtype[perm[:n_tb]] = THIRD_BODY
    rtype[perm[n_tb:n_tb + n_fo]] = FALLOFF
    n_m = int(np.count_nonzero(rtype))
    eff = rng.uniform(0.5, 3.0, (n_m, len(species)))
    lnA0 = lnA + np.log(10.0) * rng.uniform(3.0, 7.0, n_reactions)
    beta0 = beta.copy()
    Ea0 = 0.8 * Ea
    plain = rtype != FALLOFF
    lnA0[plain] = 0.0
    beta0[plain] = 0.0
    Ea0[plain] = 0.0

    return Mechanism(names=names, elements=elements, comp=comp, W=W,
                     lnA=lnA, beta=beta, Ea=Ea, reac=reac, prod=prod,
                     rtype=rtype, eff=eff, lnA0=lnA0, beta0=beta0, Ea0=Ea0,
                     fuel=1, oxidiser=0,
                     diluent=len(species) - 1 if has_n else -1, seed=seed)


R_GAS = 8.314462618  # J/(mol K)


def make_thermo(mech: Mechanism, seed: int):
    """Synthetic species thermochemistry for the energy equation: one constant
    molar heat capacity and one formation enthalpy at 298.15 K per species
    (the species enthalpy is then H_i(T) = Hf_i + cp_i (T - 298.15)).

    cp_i = R (2.5 + (atoms_i - 1)) (1 + 0.1 U(-1, 1)): 2.5 R for an atom,
    3.5 R for a diatomic, one R more per further atom. Hf_i = 150 kJ/mol
    U(-1, 1) minus 120 kJ/mol per O atom that can bind to H or C (so products
    rich in O-H and O-C bonds release heat, as in combustion); O2, N2 and H2
    are reference states with Hf = 0."""
    rng = np.random.default_rng(seed)
    comp = np.asarray(mech.comp)
    nS = comp.shape[0]
    atoms = comp.sum(axis=1)
    cp = R_GAS * (2.5 + (atoms - 1.0)) * (1.0 + 0.1 * rng.uniform(-1.0, 1.0, nS))
    col = {e: i for i, e in enumerate(mech.elements)}
    nO = comp[:, col["O"]] if "O" in col else np.zeros(nS)
    nH = comp[:, col["H"]] if "H" in col else np.zeros(nS)
    nC = comp[:, col["C"]] if "C" in col else np.zeros(nS)
    bound_O = np.minimum(nO, nH // 2 + 2 * nC)
    Hf = 1e3 * (150.0 * rng.uniform(-1.0, 1.0, nS) - 120.0 * bound_O)
    for i in range(nS):
        v = {e: int(comp[i, col[e]]) for e in mech.elements}
        if sum(v.values()) == 2 and max(v.values()) == 2 and (v.get("O") == 2 or v.get("N") == 2
                                                            or v.get("H") == 2):
            Hf[i] = 0.0  # O2, N2, H2
    return cp, Hf


def make_entropy(mech: Mechanism, seed: int):
    """Synthetic standard molar entropies at 298.15 K and 1 atm [J/(mol K)],
    for the equilibrium constants of reversible reactions: 110 + 35 (atoms - 1)
    J/(mol K) (more atoms, more degrees of freedom; H ~ 115, O2 ~ 205, H2O
    ~ 190 in real tables) times 1 + 0.1 U(-1, 1). Drawn from its own seed so
    that the heat capacities and enthalpies of make_thermo do not change."""
    rng = np.random.default_rng(seed)
    atoms = np.asarray(mech.comp).sum(axis=1)
    return (110.0 + 35.0 * (atoms - 1.0)) * (1.0 + 0.1 * rng.uniform(-1.0, 1.0, len(atoms)))


def make_reversible_mechanism(n_species: int, n_reactions: int, elements: Sequence[str],
                              tb_frac: float = 0.0, fo_frac: float = 0.0, seed: int = 0) -> Mechanism:
    """A synthetic mechanism of reversible reactions with its thermochemistry
    (cp, Hf, S0; seeds seed+3000 and seed+4000), each reaction written in its
    exothermic direction (reaction enthalpy at 298.15 K <= 0), as mechanisms
    usually list them: the fitted reverse rate is then the slow, endothermic
    one. Convert with irrev.to_irreversible before integrating."""
    m = make_mechanism(n_species, n_reactions, elements, tb_frac, fo_frac, seed)
    cp, Hf = make_thermo(m, seed + 3000)
    m = dataclasses.replace(m, cp=cp, Hf=Hf, S0=make_entropy(m, seed + 4000))
    reac, prod = m.reac.copy(), m.prod.copy()
    for j in range(n_reactions):
        dH = sum(Hf[s] for s in m.prod[j] if s >= 0) - sum(Hf[s] for s in m.reac[j] if s >= 0)
        if dH > 0:
            reac[j], prod[j] = m.prod[j], m.reac[j]
    return dataclasses.replace(m, reac=reac, prod=prod)


def make_states(mech: Mechanism, cells: int, T_range=(1000.0, 1500.0),
                T_bimodal: Optional[Sequence[Tuple[float, float]]] = None,
                p_atm=(1.0, 1.0), seed: int = 0, sort_by_T: bool = False):
    """Initial (T [K], p [Pa], Y [n_species, cells]) for ``cells`` cells.

    ``T_bimodal`` draws half the cells from each (lo, hi) interval.
    ``sort_by_T`` orders cells by temperature: neighbouring cells then hold
    similar states, the paper's "similar" ordering (Section 3). The default is
    the drawn ("random") order.
    """
    rng = np.random.default_rng(seed)
    if T_bimodal is not None:
        lo = np.array([r[0] for r in T_bimodal])
        hi = np.array([r[1] for r in T_bimodal])
        mode = rng.integers(0, len(T_bimodal), cells)
        T = rng.uniform(lo[mode], hi[mode])
    else:
        T = rng.uniform(T_range[0], T_range[1], cells)
    p = ATM * rng.uniform(p_atm[0], p_atm[1], cells)
    phi = rng.uniform(0.5, 2.0, cells)

    nS = mech.n_species
    el = mech.elements
    fv = mech.comp[mech.fuel]
    nc = fv[el.index("C")] if "C" in el else 0
    nh = fv[el.index("H")] if "H" in el else 0
    no = fv[el.index("O")] if "O" in el else 0
    o2_per_fuel = (2.0 * nc + 0.5 * nh - no) / 2.0
    moles = np.zeros((nS, cells))
    moles[mech.oxidiser] = 1.0
    moles[mech.fuel] = phi / o2_per_fuel
    if mech.diluent >= 0:
        moles[mech.diluent] = 3.76
    mass = moles * mech.W[:, None]
    Y = mass / mass.sum(axis=0, keepdims=True)

    reactive = np.ones(nS, dtype=bool)
    if mech.diluent >= 0:
        reactive[mech.diluent] = False
    w = rng.uniform(0.0, 1.0, (nS, cells)) * reactive[:, None]
    w /= w.sum(axis=0, keepdims=True)
    Y = 0.99 * Y + 0.01 * w
    Y *= 1.0 + 0.01 * rng.uniform(-1.0, 1.0, (nS, cells))
    Y /= Y.sum(axis=0, keepdims=True)
    if sort_by_T:
        idx = np.argsort(T, kind="stable")
        T, p, Y = T[idx], p[idx], Y[:, idx]
    return T, p, np.ascontiguousarray(Y)


# ---------------------------------------------------------------------------
# The five measured workloads. Seeds: mechanism 1000+n, states 2000+n.
# ---------------------------------------------------------------------------
RKCK, RKC = 0, 1
FP64, MIXED = 0, 1
GERSHGORIN, POWER = 0, 1  # RKC spectral-radius estimator

WORKLOADS = {
    "h2_9sp_rkck": dict(idx=1, n_species=9, n_reactions=38, elements=("H", "O", "N"),
                        tb=0.0, fo=0.0, cells=4096, T=(1000.0, 1500.0), p=(1.0, 1.0),
                        dt=1e-7, rtol=1e-6, atol=1e-10, method=RKCK, precision=FP64,
                        sigma=GERSHGORIN),
    "h2co_13sp_rkc": dict(idx=2, n_species=13, n_reactions=54, elements=("H", "O", "C", "N"),
                          tb=0.10, fo=0.0, cells=262144, T=(900.0, 2000.0), p=(1.0, 1.0),
                          dt=1e-6, rtol=1e-6, atol=1e-10, method=RKC, precision=FP64,
                          sigma=GERSHGORIN),
    "ch4_53sp_rkc_mixed": dict(idx=3, n_species=53, n_reactions=634,
                               elements=("H", "O", "C", "N"), tb=0.08, fo=0.04,
                               cells=131072, T=(800.0, 2200.0), p=(1.0, 20.0),
                               dt=1e-6, rtol=1e-6, atol=1e-10, method=RKC, precision=MIXED,
                               sigma=POWER),
    # The stiffness of this workload is spread by its bimodal temperatures:
    # with every activation energy at least 1e5 J/mol the cold cells'
    # reactions are frozen (2 RKC stages) while the hot cells' reach ~200
    # stages at dt = 1e-5 s, and per-cell f evaluations differ ~600-fold. With
    # the other workloads' ranges (A 1e8-1e14, Ea 0-2e5) the low-barrier
    # reactions set the stiffness at any temperature and the stages span
    # only 2-57.
    "c2h4_111sp_rkc_batched": dict(idx=4, n_species=111, n_reactions=1566,
                                   log10_A=(11.5, 17.5), Ea=(1.0e5, 3.0e5),
                                   elements=("H", "O", "C", "N"), tb=0.08, fo=0.04,
                                   cells=None, T=None, T_bimodal=((700.0, 900.0), (1800.0, 2400.0)),
                                   p=(1.0, 1.0), dt=(1e-6, 1e-5), rtol=1e-6, atol=1e-10,
                                   method=RKC, precision=FP64, sigma=POWER, instances=16,
                                   inst_cells=(512, 65536)),
}

# The constant-pressure energy equation (Eq. (E:energy)) on the first three
# workloads: same mechanisms and states, plus synthetic thermochemistry (seed
# 4000+n). RKC uses the power-method sigma: with T in the state, Gershgorin row
# sums add entries of different units (K per unit mass fraction and back) and
# overestimate the spectral radius about tenfold.
for _base, _sigma in (("h2_9sp_rkck", GERSHGORIN), ("h2co_13sp_rkc", POWER),
                      ("ch4_53sp_rkc_mixed", POWER)):
    WORKLOADS[_base + "_energy"] = dict(WORKLOADS[_base], sigma=_sigma, energy=True)


def workload_mechanism(name: str) -> Mechanism:
    w = WORKLOADS[name]
    m = make_mechanism(w["n_species"], w["n_reactions"], w["elements"],
                       w["tb"], w["fo"], seed=1000 + w["idx"],
                       log10_A=w.get("log10_A", (8.0, 14.0)), Ea_range=w.get("Ea", (0.0, 2.0e5)))
    if w.get("energy"):
        cp, Hf = make_thermo(m, 4000 + w["idx"])
        m = dataclasses.replace(m, cp=cp, Hf=Hf)
    return m


def workload_states(name: str, mech: Mechanism, cells: Optional[int] = None,
                    seed_offset: int = 0, sort_by_T: bool = False):
    w = WORKLOADS[name]
    n = w["cells"] if cells is None else cells
    return make_states(mech, n, T_range=w.get("T") or (0.0, 0.0),
                       T_bimodal=w.get("T_bimodal"), p_atm=w["p"],
                       seed=2000 + w["idx"] + seed_offset, sort_by_T=sort_by_T)


def batched_instances(name: str = "c2h4_111sp_rkc_batched", scale: float = 1.0):
    """Per-instance (cells, dt) of the batched workload: sizes log-uniform in
    [512, 65536] (seed 3004), dt alternating between the two given values.
    ``scale`` shrinks every instance (for parity tests), keeping at least 1."""
    w = WORKLOADS[name]
    rng = np.random.default_rng(3000 + w["idx"])
    lo, hi = w["inst_cells"]
    sizes = np.exp(rng.uniform(math.log(lo), math.log(hi), w["instances"]))
    sizes = np.maximum(1, np.round(sizes * scale)).astype(np.int64)
    dts = [w["dt"][i % len(w["dt"])] for i in range(w["instances"])]
    return [(int(n), float(d)) for n, d in zip(sizes, dts)]


def serve_requests(n_requests: int, seed: int = 3005, cells=(1024, 65536),
                   dt=(1e-7, 1e-5)):
    """Request stream of the serving workload: per request the mechanism key
    (13- or 53-species, p = 0.5 each), the cell count (log-uniform) and dt
    (log-uniform). Arrival times are drawn by the server from the offered
    load with the same seed."""
    rng = np.random.default_rng(seed)
    mech = np.where(rng.uniform(size=n_requests) < 0.5, "h2co_13sp_rkc", "ch4_53sp_rkc_mixed")
    n = np.round(np.exp(rng.uniform(math.log(cells[0]), math.log(cells[1]), n_requests)))
    d = np.exp(rng.uniform(math.log(dt[0]), math.log(dt[1]), n_requests))
    return [(str(m), int(c), float(t)) for m, c, t in zip(mech, n, d)]
