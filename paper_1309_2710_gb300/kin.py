"""Python binding of the C ABI in include/kin.h (argument marshalling only).

Every computation runs in libkin.so. If the library is missing this module
raises; there is no CPU fallback. Tensors are torch CUDA tensors (PyTorch
supplies device memory and streams).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np
import torch

from . import build as _build

KIN_OK, KIN_EINVAL, KIN_ENOMEM, KIN_ECUDA, KIN_EUNSUPPORTED = 0, -1, -2, -3, -4
RKCK, RKC = 0, 1
FP64, MIXED = 0, 1
CELL_OK, CELL_MAXSTEPS, CELL_HMIN, CELL_NONFINITE = 0, 1, 2, 3
STAGE_GLOBAL, STAGE_SHARED, STAGE_SHARED_ALL = 0, 1, 2
OCC_DEFAULT, OCC_HIGH = 0, 1
SIGMA_GERSHGORIN, SIGMA_POWER = 0, 1
LAYOUT_AUTO, LAYOUT_LANE, LAYOUT_WARP = 0, 1, 2
WARP_MIN_REACTIONS = 256
WARP_MAX_CELLS_PER_SM = 64
FEVAL_AUTO, FEVAL_TABLE, FEVAL_GENERATED = 0, 1, 2
GEN_MAX_SPECIES, GEN_MAX_REACTIONS, GEN_MIN_CELLS = 32, 256, 65536
MAX_INSTANCES = 128
NSTATS = 5  # per-cell statistics: f evals, accepted, rejected, sigma estimates, f evals in them


class KinError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("kin error %d: %s" % (code, msg))
        self.code = code


class MechDesc(ctypes.Structure):
    _fields_ = [("n_species", ctypes.c_int32), ("n_reactions", ctypes.c_int32),
                ("W", ctypes.c_void_p), ("lnA", ctypes.c_void_p), ("beta", ctypes.c_void_p),
                ("Ea", ctypes.c_void_p), ("reac", ctypes.c_void_p), ("prod", ctypes.c_void_p),
                ("type", ctypes.c_void_p), ("eff", ctypes.c_void_p), ("lnA0", ctypes.c_void_p),
                ("beta0", ctypes.c_void_p), ("Ea0", ctypes.c_void_p), ("cp", ctypes.c_void_p),
                ("Hf", ctypes.c_void_p)]


class Opts(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("max_steps", ctypes.c_int32), ("block_threads", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("staging", ctypes.c_int32),
                ("occupancy", ctypes.c_int32), ("sigma", ctypes.c_int32),
                ("layout", ctypes.c_int32), ("energy", ctypes.c_int32),
                ("feval", ctypes.c_int32), ("stream", ctypes.c_void_p)]


class Instance(ctypes.Structure):
    _fields_ = [("cells", ctypes.c_int64), ("T", ctypes.c_void_p), ("p", ctypes.c_void_p),
                ("Y", ctypes.c_void_p), ("ldY", ctypes.c_int64), ("dt", ctypes.c_double),
                ("rtol", ctypes.c_double), ("atol", ctypes.c_double),
                ("status", ctypes.c_void_p), ("stats", ctypes.c_void_p)]


# name -> (restype, argtypes); the header declares exactly these entry points
_SIGNATURES = {
    "kin_create_mechanism": (ctypes.c_int, [ctypes.POINTER(MechDesc), ctypes.POINTER(ctypes.c_void_p)]),
    "kin_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "kin_last_error": (ctypes.c_char_p, []),
    "kin_workspace_bytes": (ctypes.c_int64, [ctypes.c_void_p, ctypes.POINTER(Opts), ctypes.c_int64]),
    "kin_integrate": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ctypes.POINTER(Opts), ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]),
    "kin_integrate_batch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(Instance),
                                           ctypes.POINTER(Opts), ctypes.c_void_p, ctypes.c_int64]),
    "kin_rates": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int32,
                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]),
    "kin_version": (ctypes.c_char_p, []),
    "kin_generated_f_source": (ctypes.c_int64, [ctypes.POINTER(MechDesc), ctypes.c_char_p, ctypes.c_int64]),
    "kin_integrate_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                             ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                             ctypes.POINTER(Opts), ctypes.c_void_p, ctypes.c_void_p]),
    "kin_host_buffer_bytes": (ctypes.c_int64, [ctypes.c_void_p, ctypes.POINTER(Opts), ctypes.c_int64]),
    "kin_integrate_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                          ctypes.POINTER(Opts), ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_int64]),
}

_lib = None


def lib_path() -> str:
    return _build.LIB


def lib() -> ctypes.CDLL:
    """Load libkin.so. Raises if it has not been built (no fallback)."""
    global _lib
    if _lib is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError("libkin.so is not built (%s); run paper_1309_2710_gb300.build.build()" % path)
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(code: int):
    if code != KIN_OK:
        raise KinError(code, lib().kin_last_error().decode())


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream_handle(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _mech_desc(desc):
    """kin_mech_desc of a mechanism object (array attributes W, lnA, beta, Ea,
    reac, prod, rtype, eff, lnA0, beta0, Ea0 and optionally cp, Hf), and the
    arrays it points into (keep them alive while the description is used)."""
    f64 = lambda a: np.ascontiguousarray(a, dtype=np.float64)
    a = dict(W=f64(desc.W), lnA=f64(desc.lnA), beta=f64(desc.beta), Ea=f64(desc.Ea),
             reac=np.ascontiguousarray(desc.reac, dtype=np.int32),
             prod=np.ascontiguousarray(desc.prod, dtype=np.int32),
             type=np.ascontiguousarray(desc.rtype, dtype=np.int8),
             eff=f64(np.asarray(desc.eff).reshape(-1)), lnA0=f64(desc.lnA0),
             beta0=f64(desc.beta0), Ea0=f64(desc.Ea0))
    if getattr(desc, "cp", None) is not None:
        a.update(cp=f64(desc.cp), Hf=f64(desc.Hf))
    d = MechDesc(int(len(desc.W)), int(len(desc.lnA)),
                 *[a[k].ctypes.data if k in a and a[k].size else None
                   for k in ("W", "lnA", "beta", "Ea", "reac", "prod", "type", "eff",
                             "lnA0", "beta0", "Ea0", "cp", "Hf")])
    return d, a


def generated_f_source(desc) -> str:
    """The CUDA source of the generated f for a mechanism
    (kin_generated_f_source; host only)."""
    d, keep = _mech_desc(desc)
    n = lib().kin_generated_f_source(ctypes.byref(d), None, 0)
    if n < 0:
        _check(int(n))
    buf = ctypes.create_string_buffer(int(n) + 1)
    lib().kin_generated_f_source(ctypes.byref(d), buf, int(n) + 1)
    del keep
    return buf.value.decode()


class Mechanism:
    """Device-resident mechanism tables (kin_create_mechanism). `desc` has the
    array attributes W, lnA, beta, Ea, reac, prod, rtype, eff, lnA0, beta0, Ea0
    and optionally cp, Hf (e.g. a synth.Mechanism)."""

    def __init__(self, desc):
        self.n_species = int(len(desc.W))
        self.n_reactions = int(len(desc.lnA))
        d, self._arrays = _mech_desc(desc)
        self.has_thermo = "cp" in self._arrays
        h = ctypes.c_void_p()
        _check(lib().kin_create_mechanism(ctypes.byref(d), ctypes.byref(h)))
        self.handle = h

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            _check(lib().kin_destroy(self.handle))
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def workspace_bytes(self, method=RKC, precision=FP64, cells=0, block_threads=0,
                        blocks_per_sm=0, staging=STAGE_GLOBAL, occupancy=OCC_DEFAULT,
                        sigma=SIGMA_GERSHGORIN, layout=LAYOUT_AUTO, energy=0) -> int:
        o = Opts(method, precision, 0, block_threads, blocks_per_sm, staging, occupancy, sigma, layout, energy,
                 FEVAL_AUTO, None)
        n = lib().kin_workspace_bytes(self.handle, ctypes.byref(o), int(cells))
        if n < 0:
            _check(int(n))
        return int(n)

    def workspace(self, method=RKC, precision=FP64, cells=0, block_threads=0, blocks_per_sm=0,
                  device=None, staging=STAGE_GLOBAL, occupancy=OCC_DEFAULT,
                  sigma=SIGMA_GERSHGORIN, layout=LAYOUT_AUTO, energy=0) -> torch.Tensor:
        n = self.workspace_bytes(method, precision, cells, block_threads, blocks_per_sm, staging,
                                 occupancy, sigma, layout, energy)
        return torch.empty(n, dtype=torch.uint8, device=device or torch.device("cuda"))


def _check_state(mech: Mechanism, T, p, Y):
    cells = int(T.numel())
    for name, t in (("T", T), ("p", p), ("Y", Y)):
        if not (t.is_cuda and t.dtype == torch.float64):
            raise ValueError("%s must be a float64 CUDA tensor" % name)
    if p.numel() != cells or not T.is_contiguous() or not p.is_contiguous():
        raise ValueError("T and p must be contiguous with one entry per cell")
    if Y.dim() != 2 or Y.shape[0] != mech.n_species or Y.stride(1) != 1 or Y.shape[1] < cells:
        raise ValueError("Y must be [n_species, >= cells] with unit column stride")
    return cells, int(Y.stride(0))


def _check_outputs(cells: int, status, stats, cuda: bool = True):
    """The library writes `cells` status bytes and cells x NSTATS int32
    statistics: refuse smaller or mistyped buffers before the call."""
    if status is not None and (status.dtype != torch.uint8 or not status.is_contiguous()
                               or status.numel() < cells or status.is_cuda != cuda):
        raise ValueError("status must be a contiguous uint8 tensor of >= %d entries" % cells)
    if stats is not None and (stats.dtype != torch.int32 or not stats.is_contiguous()
                              or stats.numel() < cells * NSTATS or stats.is_cuda != cuda):
        raise ValueError("stats must be a contiguous int32 tensor of >= %d x %d entries"
                         % (cells, NSTATS))


@dataclass
class Cells:
    """One instance of a batched call: device tensors and its dt/tolerances."""
    T: torch.Tensor
    p: torch.Tensor
    Y: torch.Tensor
    dt: float
    rtol: float = 1e-6
    atol: float = 1e-10
    status: Optional[torch.Tensor] = None
    stats: Optional[torch.Tensor] = None


def integrate(mech: Mechanism, T, p, Y, dt, rtol, atol, method=RKC, precision=FP64,
              status=None, stats=None, workspace=None, stream=None, max_steps=0,
              block_threads=0, blocks_per_sm=0, staging=STAGE_GLOBAL, occupancy=OCC_DEFAULT,
              sigma=SIGMA_GERSHGORIN, layout=LAYOUT_AUTO, energy=0, feval=FEVAL_AUTO):
    """Integrate every cell over dt in place (kin_integrate)."""
    cells, ld = _check_state(mech, T, p, Y)
    _check_outputs(cells, status, stats)
    if workspace is None:
        workspace = mech.workspace(method, precision, cells, block_threads, blocks_per_sm, Y.device,
                                   staging, occupancy, sigma, layout, energy)
    o = Opts(method, precision, max_steps, block_threads, blocks_per_sm, staging, occupancy, sigma,
             layout, energy, feval, _stream_handle(stream))
    _check(lib().kin_integrate(mech.handle, cells, _ptr(T), _ptr(p), _ptr(Y), ld, float(dt),
                               float(rtol), float(atol), ctypes.byref(o), _ptr(status),
                               _ptr(stats), _ptr(workspace), workspace.numel()))


def make_instances(mech: Mechanism, parts: Sequence[Cells]):
    arr = (Instance * len(parts))()
    for i, c in enumerate(parts):
        cells, ld = _check_state(mech, c.T, c.p, c.Y)
        _check_outputs(cells, c.status, c.stats)
        arr[i] = Instance(cells, c.T.data_ptr(), c.p.data_ptr(), c.Y.data_ptr(), ld,
                          float(c.dt), float(c.rtol), float(c.atol),
                          None if c.status is None else c.status.data_ptr(),
                          None if c.stats is None else c.stats.data_ptr())
    return arr


def integrate_batch(mech: Mechanism, parts: Sequence[Cells], method=RKC, precision=FP64,
                    workspace=None, stream=None, max_steps=0, block_threads=0, blocks_per_sm=0,
                    staging=STAGE_GLOBAL, occupancy=OCC_DEFAULT, sigma=SIGMA_GERSHGORIN, layout=LAYOUT_AUTO, energy=0,
                    feval=FEVAL_AUTO):
    """Integrate several instances in one persistent launch (kin_integrate_batch)."""
    if not 1 <= len(parts) <= MAX_INSTANCES:
        raise ValueError("1..%d instances per launch" % MAX_INSTANCES)
    arr = make_instances(mech, parts)
    if workspace is None:
        cells = sum(int(c.T.numel()) for c in parts)
        workspace = mech.workspace(method, precision, cells, block_threads, blocks_per_sm,
                                   parts[0].Y.device, staging, occupancy, sigma, layout, energy)
    o = Opts(method, precision, max_steps, block_threads, blocks_per_sm, staging, occupancy, sigma,
             layout, energy, feval, _stream_handle(stream))
    _check(lib().kin_integrate_batch(mech.handle, len(parts), arr, ctypes.byref(o),
                                     _ptr(workspace), workspace.numel()))


def rates(mech: Mechanism, T, p, Y, precision=FP64, out=None, workspace=None, stream=None):
    """f(T, p, Y) for every cell (kin_rates); returns dY/dt with Y's layout."""
    cells, ld = _check_state(mech, T, p, Y)
    if out is None:
        out = torch.empty_strided(Y.shape, Y.stride(), dtype=Y.dtype, device=Y.device)
    if workspace is None:
        workspace = mech.workspace(RKC, precision, cells, device=Y.device, layout=LAYOUT_LANE)
    _check(lib().kin_rates(mech.handle, cells, _ptr(T), _ptr(p), _ptr(Y), ld, _ptr(out),
                           precision, _stream_handle(stream), _ptr(workspace), workspace.numel()))
    return out


def version() -> str:
    return lib().kin_version().decode()


def host_buffer(mech: Mechanism, cells: int, method=RKC, precision=FP64, device=None,
                block_threads=0, blocks_per_sm=0, staging=STAGE_GLOBAL,
                occupancy=OCC_DEFAULT, sigma=SIGMA_GERSHGORIN, layout=LAYOUT_AUTO, energy=0,
                feval=FEVAL_AUTO) -> torch.Tensor:
    """Device buffer for integrate_host (kin_host_buffer_bytes)."""
    o = Opts(method, precision, 0, block_threads, blocks_per_sm, staging, occupancy, sigma, layout, energy,
             feval, None)
    n = lib().kin_host_buffer_bytes(mech.handle, ctypes.byref(o), int(cells))
    if n < 0:
        _check(int(n))
    return torch.empty(int(n), dtype=torch.uint8, device=device or torch.device("cuda"))


def integrate_host(mech: Mechanism, T, p, Y, dt, rtol, atol, method=RKC, precision=FP64,
                   status=None, stats=None, buffer=None, stream=None, max_steps=0,
                   block_threads=0, blocks_per_sm=0, staging=STAGE_GLOBAL, occupancy=OCC_DEFAULT,
                   sigma=SIGMA_GERSHGORIN, layout=LAYOUT_AUTO, energy=0, feval=FEVAL_AUTO):
    """kin_integrate_host: T, p, Y (in place), status, stats are CPU tensors
    (pin them for asynchronous copies). Returns after enqueueing; synchronise
    the stream before reading the results."""
    cells = int(T.numel())
    for name, t in (("T", T), ("p", p), ("Y", Y)):
        if t.is_cuda or t.dtype != torch.float64:
            raise ValueError("%s must be a float64 CPU tensor" % name)
    if Y.dim() != 2 or Y.shape[0] != mech.n_species or Y.stride(1) != 1 or Y.shape[1] < cells:
        raise ValueError("Y must be [n_species, >= cells] with unit column stride")
    _check_outputs(cells, status, stats, cuda=False)
    if buffer is None:
        buffer = host_buffer(mech, cells, method, precision, None, block_threads, blocks_per_sm,
                             staging, occupancy, sigma, layout, energy, feval)
    o = Opts(method, precision, max_steps, block_threads, blocks_per_sm, staging, occupancy, sigma,
             layout, energy, feval, _stream_handle(stream))
    _check(lib().kin_integrate_host(mech.handle, cells, _ptr(T), _ptr(p), _ptr(Y), int(Y.stride(0)),
                                    float(dt), float(rtol), float(atol), ctypes.byref(o),
                                    _ptr(status), _ptr(stats), _ptr(buffer), buffer.numel()))
