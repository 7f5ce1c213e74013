// seg_tables.h -- tables of the warp layout's segmented FP32 gather (plain
// C++, no CUDA: the library builds them at mechanism upload, and a CPU test
// compiles this header on its own to check them).
//
// The isothermal f ends with the per-species production rates, Eq.
// (E:spec-rate): omega_i = sum_j nu_ij Omega_j over the nonzeros of species
// i's stoichiometric row. One warp evaluates f for one cell. Giving each lane
// whole rows leaves the warp waiting on its longest row (53 species / 634
// reactions: 115 steps of 32 lanes for 2,499 nonzeros, 68 % of the lane
// slots used). Here the nonzeros, species by species, are cut into 32 equal
// chunks of K = ceil(nnz / 32) entries, one chunk per lane; a lane sums its
// chunk in K steps and writes one partial sum per species it touches (a
// "flush"). A row cut at a chunk boundary leaves a partial on each of the
// lanes that share it; the species' owner adds them in lane order. Every
// result therefore has a fixed summation order, independent of the launch.
//
// An entry is one 32-bit word: the FP32 bits of nu_ij (an integer of the
// reaction's two reactants and two products, whose low 17 bits are zero) in
// the high half, a flush flag in bit 16 (the lane writes its running sum after
// this entry) and the reaction's position in the permuted reaction order in
// the low half: nu = float(word & 0xfffe0000), position = word & 0xffff. A
// lane's flushes go to consecutive partial slots from its first slot, and the
// slots follow the lanes in order, so the parts of a cut row sit side by side
// and no flush needs a table load. A chunk's entries of one species may come
// in any order; they are ordered so that the 32 lanes of a step read Omega
// words in distinct shared-memory banks where they can (FP32 words: bank =
// position mod 32).
#pragma once
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

namespace kin {

struct SegTables {
    int K = 0;                    // steps: entries per lane
    int nslots = 0;               // partial-sum slots, one per (lane, species) segment
    std::vector<uint32_t> ent;    // [K][32] entry words (padding: 0, nu = 0, no flush)
    std::vector<int32_t> slot0;   // [32] first partial slot of each lane
    std::vector<int32_t> part;    // [nS]: first slot << 8 | slot count; -1: empty row
};

constexpr uint32_t SEG_NU_MASK = 0xfffe0000u;
constexpr uint32_t SEG_FLUSH = 0x00010000u;
constexpr uint32_t SEG_POS_MASK = 0x0000ffffu;

// Builds the tables from the species-major rows (ptr[nS + 1]; for entry e,
// pos[e] = the reaction's permuted position and nu[e] = its net coefficient).
// Returns false where the packed form does not apply: a position above 16
// bits, a coefficient whose FP32 bits reach below bit 17, or a row spread
// over more than 255 parts.
inline bool build_seg_tables(int nS, int nR, const int* ptr, const int* pos, const double* nu,
                             SegTables& t)
{
    const int nnz = ptr[nS];
    if (nR <= 0 || nR > (int)SEG_POS_MASK + 1 || nS <= 0 || nS > (1 << 20)) return false;
    const int K = std::max(1, (nnz + 31) / 32);
    for (int e = 0; e < nnz; ++e) {
        if (pos[e] < 0 || pos[e] >= nR) return false;
        const float f = (float)nu[e];
        if ((double)f != nu[e] || f == 0.0f) return false;
        uint32_t b;
        std::memcpy(&b, &f, 4);
        if (b & ~SEG_NU_MASK) return false;
    }
    t.K = K;
    t.part.assign(nS, -1);
    t.slot0.assign(32, 0);
    // segments (lane, species, first entry, end entry), slots in lane order
    struct Seg { int lane, s, a, b; };
    std::vector<Seg> segs;
    std::vector<std::vector<int>> lane_segs(32);
    for (int l = 0; l < 32; ++l) {
        t.slot0[l] = (int)segs.size();
        const int lo = l * K, hi = std::min(nnz, lo + K);
        for (int s = 0; s < nS && lo < hi; ++s) {
            const int a = std::max(lo, ptr[s]), b = std::min(hi, ptr[s + 1]);
            if (a >= b) continue;
            const int slot = (int)segs.size();
            if (a == ptr[s]) t.part[s] = slot << 8;
            if ((t.part[s] & 0xff) == 0xff) return false;
            t.part[s] += 1;
            lane_segs[l].push_back(slot);
            segs.push_back(Seg{l, s, a, b});
        }
    }
    t.nslots = (int)segs.size();
    // entries, step by step: each lane takes from its current segment the
    // remaining entry whose Omega word falls in the least used bank of the
    // step; a segment's last entry carries the flush
    t.ent.assign((size_t)K * 32, 0u);
    std::vector<std::vector<int>> left(segs.size());
    for (size_t g = 0; g < segs.size(); ++g)
        for (int e = segs[g].a; e < segs[g].b; ++e) left[g].push_back(e);
    std::vector<size_t> cur(32, 0);
    for (int k = 0; k < K; ++k) {
        int used[32] = {0};
        for (int l = 0; l < 32; ++l) {
            if (l * K + k >= std::min(nnz, l * K + K)) continue;  // padding
            while (cur[l] < lane_segs[l].size() && left[lane_segs[l][cur[l]]].empty()) ++cur[l];
            std::vector<int>& L = left[lane_segs[l][cur[l]]];
            size_t best = 0;
            for (size_t c = 1; c < L.size(); ++c)
                if (used[pos[L[c]] % 32] < used[pos[L[best]] % 32]) best = c;
            const int e = L[best];
            L.erase(L.begin() + best);
            used[pos[e] % 32]++;
            const float f = (float)nu[e];
            uint32_t b;
            std::memcpy(&b, &f, 4);
            t.ent[(size_t)k * 32 + l] = b | (L.empty() ? SEG_FLUSH : 0u) | (uint32_t)pos[e];
        }
    }
    return true;
}

}  // namespace kin
