"""Rounding variants of the oracle, and the noise floor they measure (test
infrastructure).

The parity metric of the hot-path contract divides |Y_gpu - Y_ref| by
max(|Y_ref|, atol). Species a few atol in size carry absolute differences of
1e-18..1e-17 from rounding alone, and the finite-difference spectral radius
turns last-bit differences of f into continuous shifts of the step sequence,
so two correct FP64 implementations of the same algorithm disagree in that
metric by more than 1e-8 on the larger mechanisms. This module measures how
much: it compiles copies of the oracle that round differently but compute
the same mathematics, and reports, for given cells, the largest difference
any of them shows against the oracle itself. The GPU parity tests hold the
CUDA path to a fixed multiple of that measured floor (and to 1e-8 where the
floor is lower).

The variants (each the same formula evaluated in another legitimate order):
  fma     the oracle compiled with FMA contraction;
  expsum  Eq. (E:rxn-const) as one exp of the summed exponent,
          k = exp(ln A + beta ln T - E/(R T)), instead of three factors;
  order   the reaction sum of the production rates, the mixture sum and the
          third-body sums taken in reverse order;
  all     the three together.
"""
from __future__ import annotations

import os
import platform
import threading

import numpy as np

import oracle

_SUBS = {
    "expsum": [("k[j] = exp(m->lnA[j]) * pow(T, m->beta[j]) * exp(-m->Ea[j] / (ORC_R * T));",
                "k[j] = exp(m->lnA[j] + m->beta[j] * log(T) - m->Ea[j] / (ORC_R * T));")],
    "order": [("    for (i = 0; i < nS; i++) omega[i] = 0.0;\n    for (j = 0; j < m->nR; j++) {",
               "    for (i = 0; i < nS; i++) omega[i] = 0.0;\n    for (j = m->nR - 1; j >= 0; j--) {"),
              ("for (i = 0; i < nS; i++) sum += Y[i] / m->W[i];",
               "for (i = nS - 1; i >= 0; i--) sum += Y[i] / m->W[i];"),
              ("for (i = 0; i < nS; i++) M += a[i] * C[i];",
               "for (i = nS - 1; i >= 0; i--) M += a[i] * C[i];")],
}
VARIANTS = {"fma": ([], True), "expsum": (["expsum"], False), "order": (["order"], False),
            "all": (["expsum", "order"], True)}
_OUT = os.path.join(os.path.dirname(oracle._SRC), "_build", "variants")
_lock = threading.Lock()
_libs = {}


def variant_source(name: str) -> str:
    text = open(oracle._SRC).read()
    for key in VARIANTS[name][0]:
        for old, new in _SUBS[key]:
            assert text.count(old) == 1, "variant anchor missing: " + old
            text = text.replace(old, new)
    return text


def lib(name: str):
    """The compiled variant `name` (built once per process into oracle/_build)."""
    with _lock:
        if name not in _libs:
            os.makedirs(_OUT, exist_ok=True)
            src = os.path.join(_OUT, "kin_oracle_%s.c" % name)
            with open(src, "w") as f:
                f.write(variant_source(name))
            contract = VARIANTS[name][1]
            out = os.path.join(_OUT, "libkin_oracle_%s.so" % name)
            # FMA contraction needs the FMA instructions on x86-64; aarch64
            # has them in the base instruction set
            extra = ["-ffp-contract=fast"] if contract else []
            if contract and platform.machine() in ("x86_64", "AMD64"):
                extra.append("-mfma")
            oracle.compile_source(src, out, extra=extra)
            _libs[name] = oracle.bind(out)
        return _libs[name]


def _with_lib(L, fn):
    saved = oracle._lib
    oracle._lib = L
    try:
        return fn()
    finally:
        oracle._lib = saved


def reference(m, T, p, Y, dt, rtol, atol, method, max_steps=0, energy=False, variants=None):
    """The oracle's result for these cells and the rounding noise floor of the
    parity metric on them. Returns (Y, status, stats, floor), with T appended
    before floor when `energy`. floor is the largest |Y_v - Y_ref| /
    max(|Y_ref|, atol) over the variants, on the cells whose decision trace
    the variant reproduces (with the energy equation T counts as a component,
    relative to T)."""
    om = oracle.Mech(m)
    ref = oracle.integrate(om, T, p, Y, dt, rtol, atol, method, max_steps=max_steps, energy=energy)
    floor = 0.0
    for name in (variants or VARIANTS):
        def run():
            return oracle.integrate(oracle.Mech(m), T, p, Y, dt, rtol, atol, method,
                                    max_steps=max_steps, energy=energy)
        v = _with_lib(lib(name), run)
        same = (v[2] == ref[2]).all(axis=1)
        if not same.any():
            continue
        e = np.abs(v[0] - ref[0]) / np.maximum(np.abs(ref[0]), atol)
        floor = max(floor, float(e[:, same].max()))
        if energy:
            floor = max(floor, float((np.abs(v[4] - ref[4]) / ref[4])[same].max()))
    if energy:
        return ref[0], ref[1], ref[2], ref[4], floor
    return ref[0], ref[1], ref[2], floor
