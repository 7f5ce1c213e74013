"""Helpers for GPU-vs-oracle parity (no GPU or oracle calls at import)."""
import numpy as np


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
            max_div_frac=0.01):
    """Compare GPU and oracle states of the same cells.

    The adaptive integrators take discrete decisions (accept/reject, the
    floor in the RKC stage count, the 25-step spectral-radius refresh), so a
    last-bit difference in f can, rarely, change a cell's decision sequence
    and move its result by about the local error. Cells whose decision trace
    (f evaluations, accepted and rejected steps, spectral-radius estimates)
    matches the oracle must agree to `tol` in `tol_rel_err`; the rest must be
    a small fraction and agree to `div_tol` (default 10 rtol). Status codes
    must match. Returns a summary dict (it also reports the error relative to
    max(|Y|, atol)).
    """
    div_tol = 10 * rtol if div_tol is None else div_tol
    assert np.array_equal(st_g, st_o), "status differs: %s vs %s" % (
        np.bincount(st_g, minlength=4), np.bincount(st_o, minlength=4))
    rel = tol_rel_err(Yg, Yo, atol, rtol).max(axis=0)
    same = (sta_g == sta_o).all(axis=1)
    out = dict(cells=int(len(same)), trace_divergent=int((~same).sum()),
               max_err_same=float(rel[same].max()) if same.any() else 0.0,
               max_err_divergent=float(rel[~same].max()) if (~same).any() else 0.0,
               max_err_atol_floor=float(rel_err(Yg, Yo, atol).max()))
    assert out["max_err_same"] <= tol, out
    assert (~same).mean() <= max_div_frac, out
    assert out["max_err_divergent"] <= div_tol, out
    return out
