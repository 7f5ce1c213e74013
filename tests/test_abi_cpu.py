"""CPU checks of the C ABI library: it builds, loads, and exports every entry
point that include/kin.h declares; argument validation that runs before any
CUDA call rejects bad input. No kernel is launched here."""
import ctypes
import os
import re

import pytest

from paper_1309_2710_gb300 import build as kbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(kin_\w+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    return ctypes.CDLL(kbuild.build())


def test_header_declares_entry_points():
    names = _declared()
    for required in ("kin_create_mechanism", "kin_integrate", "kin_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_header():
    from paper_1309_2710_gb300 import kin
    assert set(kin._SIGNATURES) == _declared()


def test_create_rejects_null_without_touching_cuda(lib):
    lib.kin_create_mechanism.restype = ctypes.c_int
    lib.kin_create_mechanism.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    lib.kin_last_error.restype = ctypes.c_char_p
    assert lib.kin_create_mechanism(None, None) == -1
    assert b"non-NULL" in lib.kin_last_error()


def test_integrate_rejects_null_mechanism(lib):
    lib.kin_integrate.restype = ctypes.c_int
    assert lib.kin_integrate(None, ctypes.c_int64(1), None, None, None, ctypes.c_int64(1),
                             ctypes.c_double(1e-6), ctypes.c_double(1e-6), ctypes.c_double(1e-10),
                             None, None, None, None, ctypes.c_int64(0)) == -1


def test_version(lib):
    lib.kin_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.kin_version()


def test_binding_constants_match_the_header():
    """Every constant the binding mirrors has the header's value, and the
    binding's option struct has the header's fields in the header's order."""
    from paper_1309_2710_gb300 import kin
    src = open(os.path.join(ROOT, "include", "kin.h")).read()
    defs = {k: int(v) for k, v in re.findall(r"#define\s+(KIN_\w+)\s+\(?(-?\d+)\)?", src)}
    pairs = {"KIN_RKCK": kin.RKCK, "KIN_RKC": kin.RKC, "KIN_FP64": kin.FP64, "KIN_MIXED": kin.MIXED,
             "KIN_LAYOUT_AUTO": kin.LAYOUT_AUTO, "KIN_LAYOUT_LANE": kin.LAYOUT_LANE,
             "KIN_LAYOUT_WARP": kin.LAYOUT_WARP, "KIN_SIGMA_GERSHGORIN": kin.SIGMA_GERSHGORIN,
             "KIN_SIGMA_POWER": kin.SIGMA_POWER, "KIN_FEVAL_AUTO": kin.FEVAL_AUTO,
             "KIN_FEVAL_TABLE": kin.FEVAL_TABLE, "KIN_FEVAL_GENERATED": kin.FEVAL_GENERATED,
             "KIN_GEN_MAX_SPECIES": kin.GEN_MAX_SPECIES, "KIN_GEN_MAX_REACTIONS": kin.GEN_MAX_REACTIONS,
             "KIN_GEN_MIN_CELLS": kin.GEN_MIN_CELLS, "KIN_NSTATS": kin.NSTATS,
             "KIN_WARP_MIN_REACTIONS": kin.WARP_MIN_REACTIONS,
             "KIN_WARP_MAX_CELLS_PER_SM": kin.WARP_MAX_CELLS_PER_SM, "KIN_EUNSUPPORTED": kin.KIN_EUNSUPPORTED}
    for name, value in pairs.items():
        assert defs[name] == value, name
    plain = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    end = plain.index("} kin_opts;")
    fields = re.findall(r"\b(\w+)\s*;", plain[plain.rindex("{", 0, end) + 1:end])
    assert fields == [f for f, _ in kin.Opts._fields_]


def test_peak_probe_library_exports_its_header():
    """libkin_peaks.so exports every entry point include/kin_peaks.h declares,
    and refuses a bad argument before any CUDA call."""
    kbuild.build()
    src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "kin_peaks.h")).read(), flags=re.S)
    names = set(re.findall(r"\b(kinpk_\w+)\s*\(", src))
    assert names == {"kinpk_fma_rate", "kinpk_last_error"}
    L = ctypes.CDLL(kbuild.LIB_PEAKS)
    for name in names:
        assert hasattr(L, name), name
    from paper_1309_2710_gb300 import peaks
    ms, rate = ctypes.c_double(), ctypes.c_double()
    assert peaks.lib().kinpk_fma_rate(9, 1, 1, 32, None, ctypes.byref(ms), ctypes.byref(rate)) == -1
    assert b"precision" in peaks.lib().kinpk_last_error()
