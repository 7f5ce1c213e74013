"""Python binding of the arithmetic-peak probe (include/kin_peaks.h):
argument marshalling only; the probe runs in libkin_peaks.so."""
from __future__ import annotations

import ctypes
import os

from . import build as _build

FP64, FP32 = 0, 1
_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB_PEAKS):
            raise RuntimeError("libkin_peaks.so is not built (%s)" % _build.LIB_PEAKS)
        L = ctypes.CDLL(_build.LIB_PEAKS)
        L.kinpk_fma_rate.restype = ctypes.c_int
        L.kinpk_fma_rate.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                     ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double)]
        L.kinpk_last_error.restype = ctypes.c_char_p
        L.kinpk_last_error.argtypes = []
        _lib = L
    return _lib


def fma_rate(precision: int, iters: int, blocks_per_sm: int = 4, threads: int = 256, stream=None):
    """(kernel ms, fused multiply-adds per second) of the dependent-FMA probe
    on the current device (kinpk_fma_rate)."""
    ms, rate = ctypes.c_double(), ctypes.c_double()
    h = None if stream is None else ctypes.c_void_p(int(stream))
    rc = lib().kinpk_fma_rate(int(precision), int(iters), int(blocks_per_sm), int(threads), h,
                              ctypes.byref(ms), ctypes.byref(rate))
    if rc != 0:
        raise RuntimeError("kinpk_fma_rate: %d %s" % (rc, lib().kinpk_last_error().decode()))
    return ms.value, rate.value
