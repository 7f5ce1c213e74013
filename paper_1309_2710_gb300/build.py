"""Build the CUDA library libkin.so in-tree (sm_103a only)."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libkin.so")
# the arithmetic-peak probe behind include/kin_peaks.h: its own library, not
# part of the integrator
LIB_PEAKS = os.path.join(OUT_DIR, "libkin_peaks.so")
PEAKS_SOURCE = "peaks.cu"
SOURCES = ["kernels.cu", "abi.cu", "no_alloc.cu", "inst_rkc_f64.cu", "inst_rkc_f32.cu",
           "inst_rkck_f64.cu", "inst_rkck_f32.cu", "inst_warp_f64.cu", "inst_warp_f32.cu",
           "inst_warp_f64_hi.cu", "inst_warp_f32_hi.cu", "inst_energy_f64.cu", "inst_energy_f32.cu",
           "inst_warp_energy_f64.cu", "inst_warp_energy_f32.cu", "inst_warp_energy_f64_hi.cu",
           "inst_warp_energy_f32_hi.cu", "inst_warp_rkck_f64.cu", "inst_warp_rkck_f32.cu", "codegen.cu"]
# sources that the run-time compilation of a generated f includes, embedded
# in the library as strings: (C identifier, path)
EMBEDDED = [("kin_src_kernels", os.path.join(CSRC, "kernels.cuh")),
            ("kin_src_dev", os.path.join(CSRC, "kin_dev.cuh")),
            ("kin_src_api", os.path.join(HERE, "..", "include", "kin.h"))]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(HERE, "..", "include", "kin.h"))
    return files


def up_to_date() -> bool:
    if not os.path.exists(LIB) or not os.path.exists(LIB_PEAKS):
        return False
    t = min(os.path.getmtime(LIB), os.path.getmtime(LIB_PEAKS))
    return all(os.path.getmtime(f) <= t for f in _deps())


def write_embedded() -> str:
    """_build/kin_embedded.h: the kernel headers as raw string literals."""
    out = os.path.join(OUT_DIR, "kin_embedded.h")
    parts = ["// written by build.py: sources for the run-time compilation of a generated f\n#pragma once\n"]
    for name, path in EMBEDDED:
        text = open(path).read()
        if ")KINSRC\"" in text:
            raise RuntimeError("%s contains the raw-string delimiter" % path)
        parts.append('static const char* const %s = R"KINSRC(%s)KINSRC";\n' % (name, text))
    body = "".join(parts)
    if not os.path.exists(out) or open(out).read() != body:
        with open(out, "w") as f:
            f.write(body)
    return out


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every translation unit in parallel and link libkin.so."""
    if not force and up_to_date():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    write_embedded()
    nvcc = _nvcc()
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "-I", os.path.join(HERE, "..", "include"), "-I", OUT_DIR]
    if verbose:
        common += ["-Xptxas", "-v"]

    def compile_one(src):
        obj = os.path.join(OUT_DIR, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc] + common + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s" % (src, r.stderr))
        if verbose:
            print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(len(SOURCES) + 1) as ex:
        objs = list(ex.map(compile_one, SOURCES + [PEAKS_SOURCE]))
    for lib, parts in ((LIB, objs[:-1] + ["-ldl"]), (LIB_PEAKS, objs[-1:])):
        tmp = lib + ".%d.tmp" % os.getpid()
        cmd = [nvcc] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + parts
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n" + r.stderr)
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
