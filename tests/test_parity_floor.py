"""The rounding noise floor of the parity metric, measured on the oracle.

The variants in tests/oracle_variants.py evaluate the same formulas as the
oracle in other legitimate orders. These tests show (1) that each variant
computes the same f to rounding, so its distance from the oracle is rounding
noise and not a different method, and (2) how large that noise is in the
contract's metric |dY| / max(|Y|, atol): below 1e-8 for the 13-species
workload, above it for the 53-species one, where no FP64 implementation can
be held to 1e-8 in that metric against another."""
import numpy as np
import pytest

import oracle
from paper_1309_2710_gb300 import synth
from tests import oracle_variants as ov


@pytest.mark.parametrize("variant", list(ov.VARIANTS))
def test_variant_computes_the_same_f(variant):
    name = "ch4_53sp_rkc_mixed"
    m = synth.workload_mechanism(name)
    T, p, Y = synth.workload_states(name, m, cells=12, seed_offset=5)
    ref = [oracle.rates(oracle.Mech(m), T[c], p[c], Y[:, c]) for c in range(12)]

    def run():
        om = oracle.Mech(m)
        return [oracle.rates(om, T[c], p[c], Y[:, c]) for c in range(12)]

    got = ov._with_lib(ov.lib(variant), run)
    for a, b in zip(got, ref):
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()
        assert not np.array_equal(a, b) or variant == "fma"  # it does round differently


def test_noise_floor_small_mechanism():
    """13 species / 54 reactions, Gershgorin sigma: the variants reproduce
    every decision trace and stay within 1e-8 of the oracle."""
    name = "h2co_13sp_rkc"
    m = synth.workload_mechanism(name)
    w = synth.WORKLOADS[name]
    T, p, Y = synth.workload_states(name, m, cells=1024, seed_offset=3)
    *_, floor = ov.reference(m, T, p, Y, w["dt"], w["rtol"], w["atol"], oracle.RKC)
    print("noise floor 13/54: %.3e" % floor)
    assert 1e-13 < floor < 1e-8


def test_noise_floor_exceeds_the_target_on_the_53_species_mechanism():
    """53 species / 634 reactions: species a few atol in size differ by
    rounding-level absolute amounts that the metric's atol floor turns into
    relative errors above 1e-8, between two correct FP64 oracles."""
    name = "ch4_53sp_rkc_mixed"
    m = synth.workload_mechanism(name)
    w = synth.WORKLOADS[name]
    T, p, Y = synth.workload_states(name, m, cells=100)
    Yo, st, sta, floor = ov.reference(m, T, p, Y, w["dt"], w["rtol"], w["atol"], oracle.RKC)
    print("noise floor 53/634: %.3e" % floor)
    assert (st == 0).all()
    assert floor > 1e-8
    # ... while in the integrator's own weighting (atol/rtol floor) the same
    # variants agree to far below 1e-8
    worst = 0.0
    for v in ov.VARIANTS:
        Yv = ov._with_lib(ov.lib(v), lambda: oracle.integrate(oracle.Mech(m), T, p, Y, w["dt"], w["rtol"],
                                                              w["atol"], oracle.RKC)[0])
        worst = max(worst, float((np.abs(Yv - Yo) / np.maximum(np.abs(Yo), w["atol"] / w["rtol"])).max()))
    assert worst < 1e-9


def _arrays(n=10, species=3):
    rng = np.random.default_rng(0)
    Yo = rng.uniform(1e-3, 1.0, (species, n))
    st = np.zeros(n, np.uint8)
    sta = np.tile(np.array([[100, 40, 2, 3, 9]], np.int32), (n, 1))
    return Yo, st, sta


def test_compare_holds_trace_identical_cells_to_the_floor_bound():
    from tests.parity import compare
    Yo, st, sta = _arrays()
    Yg = Yo * (1 + 5e-9)
    out = compare(Yg, Yo, st, st, sta, sta, 1e-10, 1e-6, floor=1e-10)
    assert out["atol_floor_bound"] == 1e-8 and out["trace_divergent"] == 0
    with pytest.raises(AssertionError):  # above max(1e-8, 10 x floor)
        compare(Yo * (1 + 3e-8), Yo, st, st, sta, sta, 1e-10, 1e-6, floor=2e-9, tol=1.0)
    compare(Yo * (1 + 3e-8), Yo, st, st, sta, sta, 1e-10, 1e-6, floor=4e-9, tol=1.0)


def test_compare_mixed_splits_cells_by_their_step_decisions():
    from tests.parity import compare_mixed
    Yo, st, sta = _arrays()
    sg = sta.copy()
    sg[:, 0] += 7  # f-evaluation counts move on every cell
    Yg = Yo * (1 + 5e-6)
    out = compare_mixed(Yg, Yo, st, st, sg, sta, 1e-10, 1e-6)
    assert out["step_divergent"] == 0
    # one cell with an extra rejection may sit farther away, up to the spread
    sg[3, 2] += 1
    Yg[:, 3] = Yo[:, 3] * (1 + 5e-5)
    out = compare_mixed(Yg, Yo, st, st, sg, sta, 1e-10, 1e-6)
    assert out["step_divergent"] == 1 and out["max_err"] > 1e-5
    with pytest.raises(AssertionError):  # but not a step-identical one
        sg[3, 2] -= 1
        compare_mixed(Yg, Yo, st, st, sg, sta, 1e-10, 1e-6)
    with pytest.raises(AssertionError):  # nor anything beyond the spread
        sg[3, 2] += 1
        Yg[:, 3] = Yo[:, 3] * (1 + 5e-4)
        compare_mixed(Yg, Yo, st, st, sg, sta, 1e-10, 1e-6)
