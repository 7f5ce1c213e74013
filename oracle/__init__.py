"""Plain FP64 CPU oracle of the batched kinetics integrator (test infrastructure).

Only the tests, the smoke check and the benchmark's CPU baseline leg import
this package. The product path never does. The arithmetic lives in
``kin_oracle.c``; this module compiles it with gcc and exposes it via ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kin_oracle.c")
_OUT = os.path.join(_HERE, "_build", "libkin_oracle.so")
_lock = threading.Lock()
_lib = None

RKCK, RKC, RKC_POWER = 0, 1, 2  # method: RKC_POWER = RKC with the power-method sigma


def compile_source(src: str, out: str, extra=()) -> str:
    """gcc the oracle source ``src`` into the shared library ``out`` (no
    fast-math, no FMA contraction, so it rounds the same on x86-64 and
    aarch64). ``extra`` flags come last (the tests' rounding variants use
    them to allow contraction)."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-std=c99", "-O2", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math"] + list(extra) + [src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build`` unless it is up to date."""
    if (not force and os.path.exists(_OUT)
            and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC)):
        return _OUT
    return compile_source(_SRC, _OUT)


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            _lib = bind(build())
    return _lib


def bind(path: str) -> ctypes.CDLL:
    """Load an oracle shared library from ``path`` and declare its symbols."""
    L = ctypes.CDLL(path)
    L.orc_mech_new.restype = ctypes.c_void_p
    L.orc_mech_new.argtypes = [ctypes.c_int, ctypes.c_int] + [ctypes.c_void_p] * 11
    L.orc_mech_free.argtypes = [ctypes.c_void_p]
    L.orc_rates.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                            ctypes.c_void_p, ctypes.c_void_p]
    L.orc_rate_constants.argtypes = [ctypes.c_void_p, ctypes.c_double,
                                     ctypes.c_void_p, ctypes.c_void_p]
    L.orc_rkck_table.argtypes = [ctypes.c_void_p] * 4
    L.orc_rkc_coeffs.argtypes = [ctypes.c_int] + [ctypes.c_void_p] * 7
    L.orc_sigma.restype = ctypes.c_double
    L.orc_sigma.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                            ctypes.c_void_p, ctypes.c_double]
    L.orc_rkck_single.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_void_p, ctypes.c_double,
                                  ctypes.c_void_p, ctypes.c_void_p]
    L.orc_rkc_single.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_void_p, ctypes.c_double, ctypes.c_int,
                                 ctypes.c_void_p]
    L.orc_mech_set_thermo.argtypes = [ctypes.c_void_p] * 3
    L.orc_rates_energy.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p,
                                   ctypes.c_void_p]
    L.orc_integrate.restype = ctypes.c_int
    L.orc_integrate.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
    L.orc_trace_cell.restype = ctypes.c_int
    L.orc_trace_cell.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                 ctypes.c_int] + [ctypes.c_void_p] * 5 + [ctypes.c_int,
                                                                          ctypes.c_void_p,
                                                                          ctypes.c_void_p]
    L.orc_sigma_power.restype = ctypes.c_double
    L.orc_sigma_power.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    L.orc_has_openmp.restype = ctypes.c_int
    return L


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Mech:
    """Oracle copy of a mechanism given as plain arrays (attributes W, lnA,
    beta, Ea, reac, prod, rtype, eff, lnA0, beta0, Ea0, and optionally the
    thermochemistry cp [J/(mol K)] and Hf [J/mol] used by the energy
    equation)."""

    def __init__(self, m):
        self.n_species = int(len(m.W))
        self.n_reactions = int(len(m.lnA))
        keep = [_f64(m.W), _f64(m.lnA), _f64(m.beta), _f64(m.Ea),
                np.ascontiguousarray(m.reac, dtype=np.int32),
                np.ascontiguousarray(m.prod, dtype=np.int32),
                np.ascontiguousarray(m.rtype, dtype=np.int8),
                _f64(np.asarray(m.eff).reshape(-1)),
                _f64(m.lnA0), _f64(m.beta0), _f64(m.Ea0)]
        self._keep = keep
        self.ptr = lib().orc_mech_new(self.n_species, self.n_reactions,
                                      *[_ptr(a) for a in keep])
        self.has_thermo = getattr(m, "cp", None) is not None
        if self.has_thermo:
            cp, Hf = _f64(m.cp), _f64(m.Hf)
            lib().orc_mech_set_thermo(self.ptr, _ptr(cp), _ptr(Hf))

    def __del__(self):
        try:
            if self.ptr:
                lib().orc_mech_free(self.ptr)
                self.ptr = None
        except Exception:
            pass


def rates(om: Mech, T: float, p: float, Y) -> np.ndarray:
    """f(Y) = dY/dt at fixed T [K], p [Pa] for one cell."""
    y = _f64(Y)
    out = np.empty(om.n_species)
    lib().orc_rates(om.ptr, float(T), float(p), _ptr(y), _ptr(out))
    return out


def rates_energy(om: Mech, p: float, y) -> np.ndarray:
    """f with the energy equation: y = (Y_1..Y_nS, T) -> dy/dt for one cell."""
    y = _f64(y)
    assert y.shape == (om.n_species + 1,) and om.has_thermo
    out = np.empty_like(y)
    lib().orc_rates_energy(om.ptr, float(p), _ptr(y), _ptr(out))
    return out


def rate_constants(om: Mech, T: float):
    k = np.empty(om.n_reactions)
    k0 = np.empty(om.n_reactions)
    lib().orc_rate_constants(om.ptr, float(T), _ptr(k), _ptr(k0))
    return k, k0


def rkck_table():
    a = np.empty(6); b = np.empty(30); c = np.empty(6); cs = np.empty(6)
    lib().orc_rkck_table(_ptr(a), _ptr(b), _ptr(c), _ptr(cs))
    return a, b.reshape(6, 5), c, cs


def rkc_coeffs(s: int):
    arr = [np.zeros(s + 1) for _ in range(5)]
    w = (ctypes.c_double(), ctypes.c_double())
    lib().orc_rkc_coeffs(int(s), *[_ptr(a) for a in arr], ctypes.byref(w[0]), ctypes.byref(w[1]))
    mu, nu, mut, gt, c = arr
    return dict(mu=mu, nu=nu, mut=mut, gt=gt, c=c, w0=w[0].value, w1=w[1].value)


def sigma(om: Mech, T: float, p: float, y, atol: float) -> float:
    y = _f64(y)
    return float(lib().orc_sigma(om.ptr, float(T), float(p), _ptr(y), float(atol)))


def sigma_power(om: Mech, T: float, p: float, y, v0=None):
    """Power-method spectral radius at y. Returns (sigma, direction, f evals)."""
    y = _f64(y)
    v = np.array(v0 if v0 is not None else np.zeros_like(y), dtype=np.float64)
    it = ctypes.c_int32(0)
    if v0 is None:
        v[:] = rates(om, T, p, y)
    sig = lib().orc_sigma_power(om.ptr, float(T), float(p), _ptr(y), _ptr(v), ctypes.byref(it))
    return float(sig), v, it.value


def rkck_single(om: Mech, T, p, y, h):
    y = _f64(y)
    y5 = np.empty_like(y); err = np.empty_like(y)
    lib().orc_rkck_single(om.ptr, float(T), float(p), _ptr(y), float(h), _ptr(y5), _ptr(err))
    return y5, err


def rkc_single(om: Mech, T, p, y, h, s):
    y = _f64(y)
    out = np.empty_like(y)
    lib().orc_rkc_single(om.ptr, float(T), float(p), _ptr(y), float(h), int(s), _ptr(out))
    return out


def integrate(om: Mech, T, p, Y, dt, rtol, atol, method, max_steps=0, nthreads=0,
              energy=False):
    """Integrate every cell over dt. Y is [n_species, cells] (species-major).
    Returns (Y_new, status[cells] uint8, stats[cells, 5] int32 = nfe, accepted,
    rejected, sigma estimates, f evaluations inside them, threads used), and
    T_new with `energy` (T is then integrated with the energy equation)."""
    T = np.array(T, dtype=np.float64, copy=True); p = _f64(p)
    if energy and not om.has_thermo:
        raise ValueError("the energy equation needs the mechanism's thermochemistry")
    Yn = np.array(Y, dtype=np.float64, order="C", copy=True)
    cells = int(T.shape[0])
    assert Yn.shape == (om.n_species, cells)
    status = np.zeros(cells, dtype=np.uint8)
    stats = np.zeros((cells, 5), dtype=np.int32)
    nt = lib().orc_integrate(om.ptr, cells, _ptr(T), _ptr(p), _ptr(Yn), cells, float(dt),
                             float(rtol), float(atol), int(method), int(max_steps),
                             _ptr(status), _ptr(stats), int(nthreads), int(bool(energy)))
    if energy:
        return Yn, status, stats, nt, T
    return Yn, status, stats, nt


def trace_cell(om: Mech, T, p, y, dt, rtol, atol, method, max_steps=0, cap=100000,
               energy=False):
    """Integrate one cell recording every attempt. Returns (y_new, status,
    dict(h, err, s, accepted, sigma) arrays plus the cell's counters `stats`
    = (f evaluations, accepted, rejected, sigma estimates, f evaluations in
    them)). sigma is the spectral radius each RKC attempt took its stage
    count from (0 for RKCK). With `energy`, y = (Y_1..Y_nS, T)."""
    y = np.array(y, dtype=np.float64, copy=True)
    h = np.zeros(cap); e = np.zeros(cap); sg = np.zeros(cap)
    s = np.zeros(cap, dtype=np.int32); a = np.zeros(cap, dtype=np.int32)
    stats = np.zeros(5, dtype=np.int32)
    n = ctypes.c_int32(0)
    st = lib().orc_trace_cell(om.ptr, float(T), float(p), _ptr(y), float(dt), float(rtol),
                              float(atol), int(method), int(max_steps), int(cap), _ptr(h),
                              _ptr(e), _ptr(s), _ptr(a), ctypes.byref(n), int(bool(energy)),
                              _ptr(sg), _ptr(stats))
    k = min(n.value, cap)
    return y, st, dict(h=h[:k], err=e[:k], s=s[:k], accepted=a[:k].astype(bool), sigma=sg[:k],
                       stats=stats)
