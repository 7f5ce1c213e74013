"""The warp layout's segmented gather tables (csrc/seg_tables.h), built on
the CPU: g++ compiles the header behind a small C shim, and the tests replay
the warp's gather in numpy from the tables alone. This checks the index logic
(every nonzero visited once, every position and slot in range, partial sums
combined into the right species) before a GPU runs the tables."""
import ctypes
import shutil
import subprocess
from pathlib import Path

import numpy as np
import pytest

from paper_1309_2710_gb300 import synth

HEADER = Path(__file__).resolve().parents[1] / "paper_1309_2710_gb300" / "csrc" / "seg_tables.h"

SHIM = r"""
#include "seg_tables.h"
#include <cstring>
extern "C" int seg_build(int nS, int nR, const int* ptr, const int* pos, const double* nu,
                         int* dims, unsigned* ent, int* slot0, int* part, int cap_ent)
{
    kin::SegTables t;
    if (!kin::build_seg_tables(nS, nR, ptr, pos, nu, t)) return 0;
    dims[0] = t.K; dims[1] = t.nslots;
    if ((int)t.ent.size() > cap_ent) return -1;
    std::memcpy(ent, t.ent.data(), 4 * t.ent.size());
    std::memcpy(slot0, t.slot0.data(), 4 * 32);
    std::memcpy(part, t.part.data(), 4 * t.part.size());
    return 1;
}
"""


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("seg")
    (d / "shim.cpp").write_text(SHIM)
    so = str(d / "seg.so")
    subprocess.run(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", "-I", str(HEADER.parent), "-o", so,
                    str(d / "shim.cpp")], check=True, capture_output=True)
    L = ctypes.CDLL(so)
    L.seg_build.restype = ctypes.c_int
    return L


def rows(m, perm_seed=0):
    """Species-major rows of net coefficients (the library's CSR order:
    reactions ascending per species, zero net coefficients dropped), with a
    random reaction permutation standing in for the warp layout's order."""
    nS, nR = m.n_species, m.n_reactions
    nu = np.zeros((nR, nS))
    for j in range(nR):
        for k in m.reac[j]:
            if k >= 0:
                nu[j, k] -= 1
        for k in m.prod[j]:
            if k >= 0:
                nu[j, k] += 1
    perm_pos = np.random.default_rng(perm_seed).permutation(nR)
    ptr, pos, val, rxn = [0], [], [], []
    for i in range(nS):
        for j in range(nR):
            if nu[j, i] != 0:
                pos.append(perm_pos[j])
                val.append(nu[j, i])
                rxn.append(j)
        ptr.append(len(pos))
    return (np.array(ptr, np.int32), np.array(pos, np.int32), np.array(val, np.float64),
            np.array(rxn), perm_pos, nu)


def build(L, nS, nR, ptr, pos, nu):
    nnz = int(ptr[-1])
    cap_ent = 32 * (nnz // 32 + 2)
    dims = np.zeros(2, np.int32)
    ent = np.zeros(cap_ent, np.uint32)
    slot0 = np.zeros(32, np.int32)
    part = np.zeros(nS, np.int32)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    rc = L.seg_build(nS, nR, p(ptr), p(pos), p(nu), p(dims), p(ent), p(slot0), p(part), cap_ent)
    if rc == 0:
        return None
    assert rc == 1
    K, nslots = (int(x) for x in dims)
    return K, nslots, ent[:32 * K].reshape(K, 32), slot0, part


def replay(K, nslots, ent, slot0, part, Om, nS):
    """The warp's gather, lane by lane, as the kernel runs it (FP64 here)."""
    P = np.full(nslots, np.nan)
    visited = []
    for lane in range(32):
        slot = int(slot0[lane])
        w = 0.0
        for k in range(K):
            e = int(ent[k, lane])
            nu = np.frombuffer(np.uint32(e & 0xFFFE0000).tobytes(), np.float32)[0]
            q = e & 0xFFFF
            assert 0 <= q < len(Om)
            if nu != 0:
                visited.append((lane, k, q, float(nu)))
            w += float(nu) * Om[q]
            if e & 0x10000:
                assert 0 <= slot < nslots and np.isnan(P[slot]), "slot written twice"
                P[slot] = w
                w = 0.0
                slot += 1
        # a lane's flushes end where the next lane's slots begin
        assert slot == (slot0[lane + 1] if lane < 31 else nslots)
    out = np.zeros(nS)
    for i in range(nS):
        if part[i] < 0:
            continue
        first, cnt = part[i] >> 8, part[i] & 0xFF
        assert cnt >= 1 and first + cnt <= nslots
        s = P[first]
        for c in range(1, cnt):
            s += P[first + c]
        out[i] = s
    assert not np.isnan(P).any()  # every slot written once
    return out, visited


@pytest.mark.parametrize("name", ["ch4_53sp_rkc_mixed", "c2h4_111sp_rkc_batched", "h2co_13sp_rkc"])
def test_segmented_gather_equals_the_rows(lib, name):
    m = synth.workload_mechanism(name)
    ptr, pos, val, rxn, perm_pos, nu = rows(m)
    t = build(lib, m.n_species, m.n_reactions, ptr, pos, val)
    assert t is not None
    K, nslots, ent, slot0, part = t
    nnz = int(ptr[-1])
    assert K == -(-nnz // 32)
    assert nslots <= m.n_species + 31  # at most one cut row per chunk boundary
    Om = np.random.default_rng(1).uniform(-1, 1, m.n_reactions)
    out, visited = replay(K, nslots, ent, slot0, part, Om, m.n_species)
    # the definition: omega_i = sum_j nu_ij Omega_j, Omega at the permuted position
    want = np.array([sum(nu[j, i] * Om[perm_pos[j]] for j in range(m.n_reactions) if nu[j, i] != 0)
                     for i in range(m.n_species)])
    np.testing.assert_allclose(out, want, rtol=1e-12, atol=1e-12)
    # every nonzero exactly once, in its own species' chunk steps
    assert len(visited) == nnz
    assert sorted((q, v) for _, _, q, v in visited) == sorted(zip(pos.tolist(), val.tolist()))
    # empty rows (the inert diluent) give exactly zero
    empty = np.diff(ptr) == 0
    assert empty.any() == (part < 0).any() and (out[empty] == 0).all()


def test_balance_and_bank_spread(lib):
    """53 species / 634 reactions: 79 steps instead of the 115 that whole rows
    per lane take, and the bank order leaves fewer conflicts than the rows'
    own order."""
    m = synth.workload_mechanism("ch4_53sp_rkc_mixed")
    ptr, pos, val, *_ = rows(m)
    K, nslots, ent, slot0, part = build(lib, m.n_species, m.n_reactions, ptr, pos, val)
    assert K == 79

    def wavefronts(e):
        tot = 0
        for k in range(e.shape[0]):
            q = e[k] & 0xFFFF
            live = (e[k] & 0xFFFE0000) != 0
            qs = q[live]
            # distinct words in the same bank serialise; the same word broadcasts
            banks = {}
            for w in set(qs.tolist()):
                banks[w % 32] = banks.get(w % 32, 0) + 1
            tot += max(banks.values()) if banks else 0
        return tot / e.shape[0]

    # the same chunks in CSR order within each segment
    plain = np.zeros_like(ent)
    nnz = int(ptr[-1])
    for lane in range(32):
        for k in range(K):
            f = lane * K + k
            if f < nnz:
                b = np.float32(val[f]).view(np.uint32)
                plain[k, lane] = int(b) | int(pos[f])
    assert wavefronts(ent) < wavefronts(plain)
    print("wavefronts per step: bank order %.2f, row order %.2f" % (wavefronts(ent), wavefronts(plain)))


def test_unsupported_forms_are_refused(lib):
    ptr = np.array([0, 1, 2], np.int32)
    pos = np.array([0, 1], np.int32)
    # a coefficient whose FP32 bits need the low half (1/3)
    assert build(lib, 2, 2, ptr, pos, np.array([1.0 / 3.0, 1.0])) is None
    # a position beyond 16 bits
    assert build(lib, 2, 70000, ptr, np.array([0, 69999], np.int32), np.array([1.0, -1.0])) is None
    # a coefficient whose FP32 bits reach bit 16 (the flush flag): 1 + 2^-7
    assert build(lib, 2, 2, ptr, pos, np.array([1.0 + 2.0 ** -7, 1.0])) is None
    # a reaction position outside the reactions
    assert build(lib, 2, 2, ptr, np.array([0, 2], np.int32), np.array([1.0, -1.0])) is None
    # the ordinary form passes
    assert build(lib, 2, 2, ptr, pos, np.array([2.0, -1.0])) is not None


def _rows_from(spec, nR):
    """CSR arrays from a per-species list of (position, nu) entries."""
    ptr, pos, val = [0], [], []
    for row in spec:
        for q, v in row:
            pos.append(q)
            val.append(v)
        ptr.append(len(pos))
    return np.array(ptr, np.int32), np.array(pos, np.int32), np.array(val, np.float64)


def _edge_case(case):
    rng = np.random.default_rng(11)
    if case == "fewer_nonzeros_than_lanes":  # K = 1: most lanes only pad
        return [[(0, 1.0)], [(1, -1.0), (2, 1.0)], [], [(3, 2.0)]], 4
    if case == "one_row_over_many_lanes":  # a 250-entry row cut into 28 parts
        return [[(j, 1.0) for j in range(250)], [(j, -1.0) for j in range(10)], [(5, 2.0)]], 300
    if case == "empty_rows_between":
        spec = []
        for i in range(40):
            spec.append([] if i % 3 else [(int(q), 1.0) for q in rng.choice(90, 7, replace=False)])
        return spec, 90
    # coefficients -2..2 and rows of very different lengths
    spec = []
    for i in range(37):
        k = int(rng.integers(0, 60))
        spec.append([(int(q), float(rng.choice([-2.0, -1.0, 1.0, 2.0]))) for q in rng.choice(500, k, replace=False)])
    return spec, 500


@pytest.mark.parametrize("case", ["fewer_nonzeros_than_lanes", "one_row_over_many_lanes", "empty_rows_between",
                                  "mixed_lengths_and_coefficients"])
def test_segmented_gather_edge_cases(lib, case):
    spec, nR = _edge_case(case)
    nS = len(spec)
    ptr, pos, val = _rows_from(spec, nR)
    t = build(lib, nS, nR, ptr, pos, val)
    assert t is not None
    K, nslots, ent, slot0, part = t
    nnz = int(ptr[-1])
    assert K == max(1, -(-nnz // 32))
    assert nslots <= nS + 31
    Om = np.random.default_rng(3).uniform(-1, 1, nR)
    out, visited = replay(K, nslots, ent, slot0, part, Om, nS)
    want = np.array([sum(v * Om[q] for q, v in row) for row in spec])
    np.testing.assert_allclose(out, want, rtol=1e-12, atol=1e-12)
    assert sorted((q, v) for _, _, q, v in visited) == sorted(zip(pos.tolist(), val.tolist()))
    empty = np.diff(ptr) == 0
    assert ((part < 0) == empty).all() and (out[empty] == 0).all()
