"""Helpers for GPU-vs-oracle parity (no GPU or oracle calls at import)."""
import numpy as np

# The FP64 target in the hot-path contract's metric, |dY| / max(|Y|, atol).
CONTRACT_TOL = 1e-8
# Allowed multiple of the oracle's own rounding noise floor in that metric
# (tests/oracle_variants.py). The CUDA path differs from the oracle in more
# roundings at once than any one variant does (CUDA's exp, tree-ordered warp
# sums, the generated f's accumulation order, Newton-refined step-control
# helpers), and the integrator responds linearly to such perturbations, so
# its distance is a small multiple of the variants' distance, not a new
# scale. Fixed before the GPU measurements this bound is checked on.
FLOOR_K = 10


def rel_err(Yg, Yo, atol):
    """Per-element |Y_gpu - Y_ref| / max(|Y_ref|, atol)."""
    return np.abs(Yg - Yo) / np.maximum(np.abs(Yo), atol)


def tol_rel_err(Yg, Yo, atol, rtol):
    """Per-element error relative to the integrator's own per-species scale:
    |Y_gpu - Y_ref| / max(|Y_ref|, atol/rtol). The error test weights species
    i by atol + rtol |Y_i| (Eq. (E:rmsE)), so a species is controlled
    relatively only where |Y_i| >= atol/rtol and absolutely (to atol) below;
    this is the relative error per species under that weighting."""
    return np.abs(Yg - Yo) / np.maximum(np.abs(Yo), atol / rtol)


def compare(Yg, Yo, st_g, st_o, sta_g, sta_o, atol, rtol, tol=1e-8, div_tol=None,
            max_div_frac=0.01, floor=None):
    """Compare GPU and oracle states of the same cells.

    The adaptive integrators take discrete decisions (accept/reject, the
    floor in the RKC stage count, the 25-step spectral-radius refresh), so a
    last-bit difference in f can, rarely, change a cell's decision sequence
    and move its result by about the local error. Cells whose decision trace
    (f evaluations, accepted and rejected steps, spectral-radius estimates)
    matches the oracle must agree to `tol` in `tol_rel_err`; the rest must be
    a small fraction and agree to `div_tol` (default 10 rtol). Status codes
    must match.

    With `floor` (the oracle's rounding noise floor on the same cells, from
    tests.oracle_variants.reference), trace-identical cells must also meet
    the contract's metric rel_err: at most max(CONTRACT_TOL, FLOOR_K floor).
    Returns a summary dict with both metrics.
    """
    div_tol = 10 * rtol if div_tol is None else div_tol
    assert np.array_equal(st_g, st_o), "status differs: %s vs %s" % (
        np.bincount(st_g, minlength=4), np.bincount(st_o, minlength=4))
    rel = tol_rel_err(Yg, Yo, atol, rtol).max(axis=0)
    rel_a = rel_err(Yg, Yo, atol).max(axis=0)
    same = (sta_g == sta_o).all(axis=1)
    out = dict(cells=int(len(same)), trace_divergent=int((~same).sum()),
               max_err_same=float(rel[same].max()) if same.any() else 0.0,
               max_err_divergent=float(rel[~same].max()) if (~same).any() else 0.0,
               max_err_atol_floor=float(rel_a.max()),
               max_err_atol_floor_same=float(rel_a[same].max()) if same.any() else 0.0)
    if floor is not None:
        out["noise_floor"] = float(floor)
        out["atol_floor_bound"] = max(CONTRACT_TOL, FLOOR_K * float(floor))
    assert out["max_err_same"] <= tol, out
    assert (~same).mean() <= max_div_frac, out
    assert out["max_err_divergent"] <= div_tol, out
    if floor is not None:
        assert out["max_err_atol_floor_same"] <= out["atol_floor_bound"], out
    return out


# The spread of valid RKC solutions at rtol 1e-6 in the integrator's weighting,
# measured on the oracle: its rtol 1e-6 result differs from a converged one
# (rtol 1e-10) by up to 8.8e-5 on the 13-species workload.
VALID_SPREAD = 1e-4


def compare_mixed(Yg, Yo, st_g, st_o, sta_g, sta_o, atol, rtol, tol=1e-5, min_same_frac=0.5):
    """Compare the mixed-precision path (FP32 rates) with the FP64 oracle.

    FP32 rates perturb every error estimate a little, so the f-evaluation
    counts of every cell move, and on some cells an accept/reject decision
    flips: a second valid RKC solution, a decision apart. Cells whose
    accepted and rejected step counts equal the oracle's must agree to `tol`
    (the mixed-precision target) in the integrator's weighting; the rest to
    VALID_SPREAD; at least `min_same_frac` of the cells must take the
    oracle's decisions. Status codes must match. Returns a summary with both
    metrics."""
    assert np.array_equal(st_g, st_o), "status differs"
    e = tol_rel_err(Yg, Yo, atol, rtol).max(axis=0)
    steps = (sta_g[:, 1:3] == sta_o[:, 1:3]).all(axis=1)
    out = dict(cells=int(len(e)), step_divergent=int((~steps).sum()),
               max_err_steps_equal=float(e[steps].max()) if steps.any() else 0.0,
               max_err=float(e.max()), max_err_contract_metric=float(rel_err(Yg, Yo, atol).max()))
    assert steps.mean() >= min_same_frac, out
    assert out["max_err_steps_equal"] <= tol, out
    assert out["max_err"] <= VALID_SPREAD, out
    return out
