// abi.cu -- host side of the C ABI declared in include/kin.h: argument
// validation, mechanism packing and upload, workspace sizing, launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <climits>
#include <cstring>
#include <string>
#include <vector>

#include "codegen.h"
#include "kin_dev.cuh"
#include "seg_tables.h"

using namespace kin;

struct kin_mech {
    MechDev dev;  // device pointers into `buf`
    void* buf;
    int device;
    int nS, nR, nM;
    bool thermo;          // cp and Hf given (energy equation available)
    std::string gen_src;  // the generated f (empty when the mechanism is too large for it)
};

namespace {

thread_local char g_err[512] = "";

int fail(int code, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(cudaError_t e, const char* what)
{
    return fail(KIN_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Device pointer check: the pointer must be device (or managed) memory.
bool is_device_ptr(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

struct Grid {
    int threads, blocks;  // persistent grid
    int64_t nslots;
    int layout;           // KIN_LAYOUT_LANE or KIN_LAYOUT_WARP (resolved)
};

// Automatic layout: one warp per cell for large mechanisms (a lane's working
// set would stream from memory) and for calls too small to give every lane of
// the GPU a cell; one lane per cell otherwise.
int resolve_layout(const kin_mech* m, const kin_opts* o, int64_t cells, int nsm)
{
    if (o->layout != KIN_LAYOUT_AUTO) return o->layout;
    if (m->nR > KIN_WARP_MIN_REACTIONS) return KIN_LAYOUT_WARP;
    return cells < (int64_t)KIN_WARP_MAX_CELLS_PER_SM * nsm ? KIN_LAYOUT_WARP : KIN_LAYOUT_LANE;
}

int grid_for(const kin_mech* m, const kin_opts* o, int64_t cells, Grid* g)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != m->device) return fail(KIN_EINVAL, "mechanism lives on device %d, current device is %d", m->device, dev);
    int nsm = 0;
    e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    int maxsm = 0;
    e = cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    if (o->energy && !m->thermo)
        return fail(KIN_EUNSUPPORTED, "the energy equation needs the mechanism's cp and Hf");
    const int layout = resolve_layout(m, o, cells, nsm);
    int threads = o->block_threads > 0 ? o->block_threads : 128;
    int occ = 0, cap = 0;
    if (layout == KIN_LAYOUT_WARP) {
        if (threads % 32 != 0 || threads > 256) return fail(KIN_EINVAL, "block_threads must be a multiple of 32 and <= 256");
        const int cell_lanes = warp_cell_lanes(o->method, m->nS + o->energy);
        const size_t sm = warp_smem(m->dev, o->precision, o->energy, threads) * (32 / cell_lanes);
        if (sm > (size_t)maxsm)
            return fail(KIN_EUNSUPPORTED, "warp layout needs %zu bytes of shared memory per block (max %d)", sm, maxsm);
        const int nV = m->nS + o->energy;
        if (o->method == KIN_RKCK) {
            e = o->precision == KIN_MIXED ? occ_warp_rkck_f32(m->dev, nV, o->energy, threads, &occ)
                                          : occ_warp_rkck_f64(m->dev, nV, o->energy, threads, &occ);
        } else {
            using OccFn = cudaError_t (*)(const MechDev&, int, int, int*);
            // [energy][precision][occupancy]
            static const OccFn fns[2][2][2] = {
                {{occ_warp_f64_o0, occ_warp_f64_o1}, {occ_warp_f32_o0, occ_warp_f32_o1}},
                {{occ_warp_f64_en_o0, occ_warp_f64_en_o1}, {occ_warp_f32_en_o0, occ_warp_f32_en_o1}}};
            e = fns[o->energy][o->precision == KIN_MIXED][o->occupancy ? 1 : 0](m->dev, nV, threads, &occ);
        }
        cap = occ;  // as many as fit
    } else {
        if (threads % 32 != 0 || threads > 128) return fail(KIN_EINVAL, "block_threads must be a multiple of 32 and <= 128");
        const int stg = o->energy ? KIN_STAGE_GLOBAL : o->staging;  // energy: nothing to stage
        if (stg > 0 && smem_bytes(m->dev, o->precision, threads, stg) > (size_t)maxsm)
            return fail(KIN_EUNSUPPORTED, "shared-memory staging needs %zu bytes per block (max %d)",
                        smem_bytes(m->dev, o->precision, threads, stg), maxsm);
        e = integrate_occupancy(m->dev, o->method, o->precision, stg, o->occupancy, o->energy, threads,
                                &occ);
        cap = (o->occupancy ? 768 : 512) / threads;
    }
    if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
    if (occ < 1) return fail(KIN_EUNSUPPORTED, "kernel does not fit on an SM with these options");
    int bps = o->blocks_per_sm;
    if (bps <= 0) bps = std::max(1, std::min(occ, cap));
    if (bps > occ) return fail(KIN_EINVAL, "blocks_per_sm %d exceeds the %d blocks that fit per SM", bps, occ);
    g->threads = threads;
    g->blocks = nsm * bps;
    g->nslots = (int64_t)g->blocks * threads;
    g->layout = layout;
    return KIN_OK;
}

// Workspace bytes; the warp layout keeps no per-lane arrays.
int64_t ws_bytes(const kin_mech* m, const kin_opts* o, const Grid& g, int64_t cells)
{
    const int sig = o->method == KIN_RKC ? o->sigma : KIN_SIGMA_GERSHGORIN;
    return ws_layout(m->dev, o->precision, sig, o->energy, g.layout == KIN_LAYOUT_WARP ? 0 : g.nslots,
                     cells).total;
}

int check_opts(const kin_opts* o)
{
    if (!o) return fail(KIN_EINVAL, "opts is NULL");
    if (o->method != KIN_RKCK && o->method != KIN_RKC) return fail(KIN_EINVAL, "unknown method %d", o->method);
    if (o->precision != KIN_FP64 && o->precision != KIN_MIXED)
        return fail(KIN_EINVAL, "unknown precision %d", o->precision);
    if (o->staging != KIN_STAGE_GLOBAL && o->staging != KIN_STAGE_SHARED &&
        o->staging != KIN_STAGE_SHARED_ALL)
        return fail(KIN_EINVAL, "unknown staging %d", o->staging);
    if (o->occupancy != KIN_OCC_DEFAULT && o->occupancy != KIN_OCC_HIGH)
        return fail(KIN_EINVAL, "unknown occupancy %d", o->occupancy);
    if (o->sigma != KIN_SIGMA_GERSHGORIN && o->sigma != KIN_SIGMA_POWER)
        return fail(KIN_EINVAL, "unknown sigma estimator %d", o->sigma);
    if (o->layout != KIN_LAYOUT_AUTO && o->layout != KIN_LAYOUT_LANE && o->layout != KIN_LAYOUT_WARP)
        return fail(KIN_EINVAL, "unknown layout %d", o->layout);
    if (o->energy != 0 && o->energy != 1) return fail(KIN_EINVAL, "energy must be 0 or 1");
    if (o->feval != KIN_FEVAL_AUTO && o->feval != KIN_FEVAL_TABLE && o->feval != KIN_FEVAL_GENERATED)
        return fail(KIN_EINVAL, "unknown feval %d", o->feval);
    return KIN_OK;
}

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

}  // namespace

int kin::set_last_error(int code, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

int kin::noalloc_opts(const kin_mech* m, const kin_opts* in, int64_t cells, int64_t cap,
                      kin_opts* out)
{
    g_err[0] = 0;
    if (!m) return fail(KIN_EINVAL, "mechanism is NULL");
    if (cells < 0) return fail(KIN_EINVAL, "cells < 0");
    int rc = check_opts(in);
    if (rc) return rc;
    kin_opts o = *in;
    // Never compile here: NVRTC and loading the compiled library allocate
    // device memory. The generated f runs only where an earlier call loaded
    // it on this device; otherwise the automatic choice falls back to the
    // tables and a forced one is refused.
    if (o.feval != KIN_FEVAL_TABLE && (m->gen_src.empty() || !gen_loaded(m->device, m->gen_src))) {
        if (o.feval == KIN_FEVAL_GENERATED)
            return fail(KIN_EUNSUPPORTED,
                        "kin_integrate_noalloc: the generated f of this mechanism is not loaded on "
                        "device %d (a kin_integrate call with KIN_FEVAL_GENERATED compiles and loads "
                        "it, which allocates)", m->device);
        o.feval = KIN_FEVAL_TABLE;
    }
    Grid g;
    rc = grid_for(m, &o, cells, &g);  // resolves blocks_per_sm = 0 to "as many as fit"
    if (rc) return rc;
    int nsm = 1;
    cudaError_t e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, m->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    int64_t need = 0;
    for (int bps = g.blocks / nsm; bps >= 1; --bps) {
        o.blocks_per_sm = bps;
        rc = grid_for(m, &o, cells, &g);
        if (rc) return rc;
        need = ws_bytes(m, &o, g, cells);
        if (need <= cap) {
            *out = o;
            return KIN_OK;
        }
    }
    return fail(KIN_ENOMEM,
                "kin_integrate_noalloc: %lld cells need %lld bytes of working memory even at one "
                "block per SM, more than the %lld-byte fixed array",
                (long long)cells, (long long)need, (long long)cap);
}

extern "C" {

const char* kin_last_error(void) { return g_err; }

const char* kin_version(void) { return "kin 0.3 (sm_103a)"; }

int64_t kin_generated_f_source(const kin_mech_desc* d, char* buf, int64_t cap)
{
    g_err[0] = 0;
    if (!d) return fail(KIN_EINVAL, "desc is NULL");
    if (cap < 0 || (cap > 0 && !buf)) return fail(KIN_EINVAL, "buf is NULL or cap < 0");
    const int nS = d->n_species, nR = d->n_reactions;
    if (nS < 1 || nS > KIN_MAX_SPECIES || nR < 0 || nR > KIN_MAX_REACTIONS)
        return fail(KIN_EINVAL, "n_species %d / n_reactions %d out of range", nS, nR);
    if (!gen_eligible(nS, nR))
        return fail(KIN_EUNSUPPORTED, "the generated f covers at most %d species and %d reactions",
                    KIN_GEN_MAX_SPECIES, KIN_GEN_MAX_REACTIONS);
    if (!d->W || (nR > 0 && (!d->reac || !d->prod || !d->type)))
        return fail(KIN_EINVAL, "W, reac, prod and type must be non-NULL");
    int rows = 0;
    for (int i = 0; i < nS; ++i)
        if (!finite_pos(d->W[i])) return fail(KIN_EINVAL, "W[%d] must be finite and > 0", i);
    for (int j = 0; j < nR; ++j) {
        const int t = d->type[j];
        if (t != KIN_RXN_PLAIN && t != KIN_RXN_THIRD_BODY && t != KIN_RXN_FALLOFF)
            return fail(KIN_EINVAL, "reaction %d: unknown type %d", j, t);
        for (int k = 0; k < 2; ++k)
            if (d->reac[2 * j + k] < -1 || d->reac[2 * j + k] >= nS || d->prod[2 * j + k] < -1 ||
                d->prod[2 * j + k] >= nS)
                return fail(KIN_EINVAL, "reaction %d: species index out of range", j);
        rows += t != KIN_RXN_PLAIN;
    }
    if (rows > 0 && !d->eff) return fail(KIN_EINVAL, "eff is NULL but %d reactions need efficiencies", rows);
    for (int64_t k = 0; k < (int64_t)rows * nS; ++k)
        if (!std::isfinite(d->eff[k])) return fail(KIN_EINVAL, "non-finite efficiency");
    if ((d->cp != nullptr) != (d->Hf != nullptr)) return fail(KIN_EINVAL, "give both cp and Hf, or neither");
    for (int i = 0; d->cp && i < nS; ++i)
        if (!finite_pos(d->cp[i]) || !std::isfinite(d->Hf[i]))
            return fail(KIN_EINVAL, "species %d: cp must be finite and > 0, Hf finite", i);
    if (nR > 0 && (!d->lnA || !d->beta || !d->Ea)) return fail(KIN_EINVAL, "Arrhenius arrays must be non-NULL");
    for (int j = 0; j < nR; ++j)
        if (d->type[j] == KIN_RXN_FALLOFF && (!d->lnA0 || !d->beta0 || !d->Ea0))
            return fail(KIN_EINVAL, "falloff reaction %d needs lnA0, beta0, Ea0", j);
    const std::string src = gen_f_source(d);
    if (cap > 0) {
        const int64_t n = std::min<int64_t>(cap - 1, (int64_t)src.size());
        memcpy(buf, src.data(), (size_t)n);
        buf[n] = 0;
    }
    return (int64_t)src.size();
}

int kin_create_mechanism(const kin_mech_desc* d, kin_mech** out)
{
    g_err[0] = 0;
    if (!d || !out) return fail(KIN_EINVAL, "desc and out must be non-NULL");
    *out = nullptr;
    const int nS = d->n_species, nR = d->n_reactions;
    if (nS < 1 || nS > KIN_MAX_SPECIES) return fail(KIN_EINVAL, "n_species %d out of range", nS);
    if (nR < 0 || nR > KIN_MAX_REACTIONS) return fail(KIN_EINVAL, "n_reactions %d out of range", nR);
    if (!d->W) return fail(KIN_EINVAL, "W is NULL");
    if (nR > 0 && (!d->lnA || !d->beta || !d->Ea || !d->reac || !d->prod || !d->type))
        return fail(KIN_EINVAL, "reaction arrays must be non-NULL");
    for (int i = 0; i < nS; ++i)
        if (!finite_pos(d->W[i])) return fail(KIN_EINVAL, "W[%d] must be finite and > 0", i);

    std::vector<Rxn> rxn(nR);
    std::vector<double> EaR(nR), lnA0(nR, 0.0), beta0(nR, 0.0), Ea0R(nR, 0.0);
    std::vector<std::vector<std::pair<int, double>>> bySp(nS);
    int nM = 0, nFO = 0;
    for (int j = 0; j < nR; ++j) {
        const int t = d->type[j];
        if (t != KIN_RXN_PLAIN && t != KIN_RXN_THIRD_BODY && t != KIN_RXN_FALLOFF)
            return fail(KIN_EINVAL, "reaction %d: unknown type %d", j, t);
        if (!std::isfinite(d->lnA[j]) || !std::isfinite(d->beta[j]) || !std::isfinite(d->Ea[j]))
            return fail(KIN_EINVAL, "reaction %d: non-finite Arrhenius parameter", j);
        int r[2] = {d->reac[2 * j], d->reac[2 * j + 1]};
        int q[2] = {d->prod[2 * j], d->prod[2 * j + 1]};
        for (int k = 0; k < 2; ++k) {
            if (r[k] < -1 || r[k] >= nS) return fail(KIN_EINVAL, "reaction %d: reactant index %d", j, r[k]);
            if (q[k] < -1 || q[k] >= nS) return fail(KIN_EINVAL, "reaction %d: product index %d", j, q[k]);
        }
        rxn[j] = Rxn{(int16_t)r[0], (int16_t)r[1], (int16_t)t, 0, t != KIN_RXN_PLAIN ? nM : -1,
                     t == KIN_RXN_FALLOFF ? nFO : -1};
        if (t != KIN_RXN_PLAIN) ++nM;
        if (t == KIN_RXN_FALLOFF) ++nFO;
        EaR[j] = d->Ea[j] / R_GAS;
        if (t == KIN_RXN_FALLOFF) {
            if (!d->lnA0 || !d->beta0 || !d->Ea0)
                return fail(KIN_EINVAL, "falloff reaction %d needs lnA0, beta0, Ea0", j);
            if (!std::isfinite(d->lnA0[j]) || !std::isfinite(d->beta0[j]) || !std::isfinite(d->Ea0[j]))
                return fail(KIN_EINVAL, "reaction %d: non-finite low-pressure parameter", j);
            lnA0[j] = d->lnA0[j];
            beta0[j] = d->beta0[j];
            Ea0R[j] = d->Ea0[j] / R_GAS;
        }
        // net coefficients nu'' - nu' per species of this reaction
        int sp[4] = {q[0], q[1], r[0], r[1]};
        double c[4] = {1, 1, -1, -1};
        for (int a = 0; a < 4; ++a) {
            if (sp[a] < 0) continue;
            auto& v = bySp[sp[a]];
            if (!v.empty() && v.back().first == j) v.back().second += c[a];
            else v.push_back({j, c[a]});
        }
    }
    if (nM > 0 && !d->eff) return fail(KIN_EINVAL, "eff is NULL but %d reactions need efficiencies", nM);
    for (int64_t k = 0; k < (int64_t)nM * nS; ++k)
        if (!std::isfinite(d->eff[k])) return fail(KIN_EINVAL, "non-finite efficiency");
    std::vector<int> ptr(nS + 1, 0), crx;
    std::vector<double> cnu;
    for (int i = 0; i < nS; ++i) {
        for (auto& pr : bySp[i])
            if (pr.second != 0.0) {  // a species on both sides with equal count cancels
                crx.push_back(pr.first);
                cnu.push_back(pr.second);
            }
        ptr[i + 1] = (int)crx.size();
    }
    const int nnz = (int)crx.size();

    // one device buffer, 256-byte aligned sub-arrays
    std::vector<char> host;
    auto put = [&](const void* src, size_t bytes) {
        size_t off = (host.size() + 255) / 256 * 256;
        host.resize(off + bytes);
        if (bytes) memcpy(host.data() + off, src, bytes);
        return off;
    };
    std::vector<double> invW(nS);
    std::vector<float> invW32(nS), W32(nS), nu32(cnu.begin(), cnu.end());
    for (int i = 0; i < nS; ++i) {
        invW[i] = 1.0 / d->W[i];
        invW32[i] = (float)invW[i];
        W32[i] = (float)d->W[i];
    }
    std::vector<float> eff32((size_t)nM * nS);
    for (size_t k = 0; k < eff32.size(); ++k) eff32[k] = (float)d->eff[k];
    const size_t oW = put(d->W, 8 * nS), oIW = put(invW.data(), 8 * nS), oIW32 = put(invW32.data(), 4 * nS);
    const size_t oW32 = put(W32.data(), 4 * nS);
    const size_t oLA = put(d->lnA, 8 * nR), oB = put(d->beta, 8 * nR), oE = put(EaR.data(), 8 * nR);
    const size_t oLA0 = put(lnA0.data(), 8 * nR), oB0 = put(beta0.data(), 8 * nR), oE0 = put(Ea0R.data(), 8 * nR);
    const size_t oRx = put(rxn.data(), sizeof(Rxn) * nR);
    // warp layout: reactions permuted plain, third-body, falloff (each in
    // reaction order, so falloff ordinals keep their order); efficiency rows
    // transposed to [species][non-plain reaction in permutation order]
    std::vector<int> perm, pos(nR);
    for (int t = KIN_RXN_PLAIN; t <= KIN_RXN_FALLOFF; ++t)
        for (int j = 0; j < nR; ++j)
            if (rxn[j].type == t) perm.push_back(j);
    std::vector<Rxn> rxnp(nR);
    const int nPlain = nR - nM;
    for (int q = 0; q < nR; ++q) {
        pos[perm[q]] = q;
        rxnp[q] = rxn[perm[q]];
        rxnp[q].row = rxnp[q].type != KIN_RXN_PLAIN ? q - nPlain : -1;
    }
    std::vector<int> crxp(nnz);
    for (int e2 = 0; e2 < nnz; ++e2) crxp[e2] = pos[crx[e2]];
    std::vector<double> effV64((size_t)(nS + 1) / 2 * nM * 2, 0.0);
    std::vector<float> effV32((size_t)(nS + 3) / 4 * nM * 4, 0.0f);
    for (int q = nPlain; q < nR; ++q)
        for (int k = 0; k < nS; ++k) {
            const double a = d->eff[(size_t)rxn[perm[q]].row * nS + k];
            const int row = q - nPlain;
            effV64[((size_t)(k / 2) * nM + row) * 2 + k % 2] = a;
            effV32[((size_t)(k / 4) * nM + row) * 4 + k % 4] = (float)a;
        }
    // the warp f derives a reaction's efficiency row and falloff ordinal from
    // its permutation position
    std::vector<uint32_t> rxw(nR);
    for (int q = 0; q < nR; ++q) {
        const Rxn& x = rxnp[q];
        if ((x.type != KIN_RXN_PLAIN) != (q >= nPlain) || (x.type != KIN_RXN_PLAIN && x.row != q - nPlain) ||
            (x.type == KIN_RXN_FALLOFF) != (q >= nR - nFO) || (x.type == KIN_RXN_FALLOFF && x.fo != q - (nR - nFO)))
            return fail(KIN_EUNSUPPORTED, "reaction permutation out of order at %d", q);
        rxw[q] = (uint32_t)(x.r0 + 1) | ((uint32_t)(x.r1 + 1) << 16);
    }
    const size_t oPerm = put(perm.data(), 4 * nR), oRxp = put(rxnp.data(), sizeof(Rxn) * nR);
    const size_t oRxw = put(rxw.data(), 4 * nR);
    const size_t oCrxp = put(crxp.data(), 4 * nnz);
    const size_t oEffV64 = put(effV64.data(), 8 * effV64.size()), oEffV32 = put(effV32.data(), 4 * effV32.size());
    const size_t oPtr = put(ptr.data(), 4 * (nS + 1)), oCrx = put(crx.data(), 4 * nnz);
    const size_t oNu = put(cnu.data(), 8 * nnz), oNu32 = put(nu32.data(), 4 * nnz);
    // the species' molar mass folded into its row (a common factor of the row)
    std::vector<double> cnuW(nnz);
    std::vector<float> nuW32(nnz);
    for (int i = 0; i < nS; ++i)
        for (int e2 = ptr[i]; e2 < ptr[i + 1]; ++e2) {
            cnuW[e2] = cnu[e2] * d->W[i];
            nuW32[e2] = (float)cnuW[e2];
        }
    const size_t oNuW = put(cnuW.data(), 8 * nnz), oNuW32 = put(nuW32.data(), 4 * nnz);
    // ELL copies of the gather entries for the warp layout's 32 lanes
    int ell_base[ELL_SLOTS] = {0};
    int ell_n = 0;
    for (int r = 0; r * 32 < nS; ++r) {
        int len = 0;
        for (int i = 32 * r; i < std::min(nS, 32 * r + 32); ++i) len = std::max(len, ptr[i + 1] - ptr[i]);
        ell_base[r] = ell_n;
        ell_n += 32 * len;
    }
    // Each species' entries are ordered step by step so that the lanes of a
    // step read Omega words in distinct shared-memory banks where they can:
    // for FP32 words the bank is the position mod 32 across the warp; for
    // FP64 words, read by half-warps, the position mod 16 within each half.
    // A greedy pass gives each lane, in turn, its remaining entry in the
    // least used bank of the step. Only the summation order of a row
    // follows from this; its entries do not change.
    std::vector<int> ord32(nnz), ord64(nnz);
    auto order_rows = [&](std::vector<int>& ord, int banks, int group) {
        for (int r = 0; r * 32 < nS; ++r) {
            std::vector<std::vector<int>> left(32);
            int len = 0;
            for (int l = 0; l < 32 && 32 * r + l < nS; ++l) {
                const int i = 32 * r + l;
                for (int e2 = ptr[i]; e2 < ptr[i + 1]; ++e2) left[l].push_back(e2);
                len = std::max(len, ptr[i + 1] - ptr[i]);
            }
            for (int k = 0; k < len; ++k) {
                std::vector<int> used(2 * banks, 0);
                for (int l = 0; l < 32; ++l) {
                    if (left[l].empty()) continue;
                    const int gbase = (l / group) * banks;
                    size_t best = 0;
                    for (size_t c = 1; c < left[l].size(); ++c)
                        if (used[gbase + crxp[left[l][c]] % banks] < used[gbase + crxp[left[l][best]] % banks])
                            best = c;
                    const int e2 = left[l][best];
                    left[l].erase(left[l].begin() + best);
                    used[gbase + crxp[e2] % banks]++;
                    ord[ptr[32 * r + l] + k] = e2;
                }
            }
        }
    };
    order_rows(ord32, 32, 32);
    order_rows(ord64, 16, 16);
    std::vector<CsrW32> ell32(ell_n, CsrW32{0.0f, 0});
    std::vector<CsrW64> ell64(ell_n, CsrW64{0.0, 0, 0});
    for (int i = 0; i < nS; ++i)
        for (int k = 0; k < ptr[i + 1] - ptr[i]; ++k) {
            const int at = ell_base[i / 32] + 32 * k + i % 32;
            const int a = ord32[ptr[i] + k], b = ord64[ptr[i] + k];
            ell32[at] = CsrW32{nuW32[a], crxp[a]};
            ell64[at] = CsrW64{cnuW[b], crxp[b], 0};
        }
    const size_t oEll32 = put(ell32.data(), sizeof(CsrW32) * ell_n);
    const size_t oEll64 = put(ell64.data(), sizeof(CsrW64) * ell_n);
    // the segmented FP32 gather of the 32-lane isothermal f, where the packed
    // entries apply and its partial sums fit in the FP32 half of the warp's
    // shared words, past C and Omega
    SegTables seg;
    const int group_floats = 2 * ((nS + nR + 3) & ~3);
    const bool use_seg = build_seg_tables(nS, nR, ptr.data(), crxp.data(), cnu.data(), seg) &&
                         nS + nR + seg.nslots <= group_floats;
    const size_t oSegE = use_seg ? put(seg.ent.data(), 4 * seg.ent.size()) : 0;
    const size_t oSegF = use_seg ? put(seg.slot0.data(), 4 * seg.slot0.size()) : 0;
    const size_t oSegP = use_seg ? put(seg.part.data(), 4 * seg.part.size()) : 0;
    const size_t oEff = put(d->eff, 8 * (size_t)nM * nS), oEff32 = put(eff32.data(), 4 * (size_t)nM * nS);
    // thermochemistry for the energy equation: cp, cp/W, Hf
    const bool thermo = d->cp && d->Hf;
    if ((d->cp != nullptr) != (d->Hf != nullptr)) return fail(KIN_EINVAL, "give both cp and Hf, or neither");
    std::vector<double> cpW(thermo ? nS : 0);
    for (int i = 0; thermo && i < nS; ++i) {
        if (!finite_pos(d->cp[i])) return fail(KIN_EINVAL, "cp[%d] must be finite and > 0", i);
        if (!std::isfinite(d->Hf[i])) return fail(KIN_EINVAL, "Hf[%d] must be finite", i);
        cpW[i] = d->cp[i] / d->W[i];
    }
    const size_t oCp = thermo ? put(d->cp, 8 * nS) : 0, oCpW = thermo ? put(cpW.data(), 8 * nS) : 0;
    const size_t oHf = thermo ? put(d->Hf, 8 * nS) : 0;
    const size_t oTab = put(nullptr, 0);
    const size_t tabBytes = sizeof(double) * RKC_TAB_S * RKC_TAB_S * RKC_TAB_W;
    host.resize(oTab + tabBytes, 0);

    kin_mech* m = new (std::nothrow) kin_mech();
    if (!m) return fail(KIN_ENOMEM, "host allocation failed");
    cudaError_t e = cudaGetDevice(&m->device);
    if (e != cudaSuccess) { delete m; return cuda_fail(e, "cudaGetDevice"); }
    e = cudaMalloc(&m->buf, host.size());
    if (e != cudaSuccess) { delete m; cudaGetLastError(); return fail(KIN_ENOMEM, "cudaMalloc(%zu): %s", host.size(), cudaGetErrorString(e)); }
    e = cudaMemcpy(m->buf, host.data(), host.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { cudaFree(m->buf); delete m; return cuda_fail(e, "cudaMemcpy"); }
    char* b = (char*)m->buf;
    MechDev& M = m->dev;
    M.nS = nS; M.nR = nR; M.nM = nM; M.nFO = nFO; M.nnz = nnz;
    M.W = (const double*)(b + oW); M.invW = (const double*)(b + oIW); M.invW32 = (const float*)(b + oIW32);
    M.W32 = (const float*)(b + oW32);
    M.lnA = (const double*)(b + oLA); M.beta = (const double*)(b + oB); M.EaR = (const double*)(b + oE);
    M.lnA0 = (const double*)(b + oLA0); M.beta0 = (const double*)(b + oB0); M.Ea0R = (const double*)(b + oE0);
    M.rxn = (const Rxn*)(b + oRx);
    M.rxn_perm = (const int*)(b + oPerm);
    M.rxnp = (const Rxn*)(b + oRxp);
    M.csrp_rxn = (const int*)(b + oCrxp);
    M.ell32 = (const CsrW32*)(b + oEll32);
    M.ell64 = (const CsrW64*)(b + oEll64);
    for (int r = 0; r < ELL_SLOTS; ++r) M.ell_base[r] = ell_base[r];
    M.seg_ent = use_seg ? (const uint32_t*)(b + oSegE) : nullptr;
    M.seg_slot0 = use_seg ? (const int32_t*)(b + oSegF) : nullptr;
    M.seg_part = use_seg ? (const int32_t*)(b + oSegP) : nullptr;
    M.seg_K = use_seg ? seg.K : 0;
    M.effV64 = (const double*)(b + oEffV64);
    M.effV32 = (const float*)(b + oEffV32);
    M.rxw = (const uint32_t*)(b + oRxw);
    M.csr_ptr = (const int*)(b + oPtr); M.csr_rxn = (const int*)(b + oCrx);
    M.csr_nu = (const double*)(b + oNu); M.csr_nu32 = (const float*)(b + oNu32);
    M.csr_nuW = (const double*)(b + oNuW); M.csr_nuW32 = (const float*)(b + oNuW32);
    M.eff = (const double*)(b + oEff); M.eff32 = (const float*)(b + oEff32);
    M.rkc = (const double*)(b + oTab);
    M.cp = thermo ? (const double*)(b + oCp) : nullptr;
    M.cpW = thermo ? (const double*)(b + oCpW) : nullptr;
    M.Hf = thermo ? (const double*)(b + oHf) : nullptr;
    m->nS = nS; m->nR = nR; m->nM = nM;
    m->thermo = thermo;
    if (gen_eligible(nS, nR)) m->gen_src = gen_f_source(d);
    e = launch_rkc_table((double*)(b + oTab), 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) { cudaFree(m->buf); delete m; return cuda_fail(e, "RKC table"); }
    *out = m;
    return KIN_OK;
}

int kin_destroy(kin_mech* m)
{
    g_err[0] = 0;
    if (!m) return KIN_OK;
    cudaError_t e = cudaFree(m->buf);
    delete m;
    return e == cudaSuccess ? KIN_OK : cuda_fail(e, "cudaFree");
}

int64_t kin_workspace_bytes(const kin_mech* m, const kin_opts* o, int64_t cells)
{
    g_err[0] = 0;
    if (!m) return fail(KIN_EINVAL, "mechanism is NULL");
    if (cells < 0) return fail(KIN_EINVAL, "cells < 0");
    int rc = check_opts(o);
    if (rc) return rc;
    Grid g;
    rc = grid_for(m, o, cells, &g);
    if (rc) return rc;
    return ws_bytes(m, o, g, cells);
}

int kin_integrate_batch(const kin_mech* m, int32_t n, const kin_instance* inst, const kin_opts* o,
                        void* ws, int64_t ws_size)
{
    g_err[0] = 0;
    if (!m) return fail(KIN_EINVAL, "mechanism is NULL");
    int rc = check_opts(o);
    if (rc) return rc;
    if (n < 1 || n > KIN_MAX_INSTANCES) return fail(KIN_EINVAL, "n_instances %d out of range [1, %d]", n, KIN_MAX_INSTANCES);
    if (!inst) return fail(KIN_EINVAL, "instances is NULL");
    // ~10 KB of launch parameters: built on the heap, copied by the launch
    Launch* Lp = new (std::nothrow) Launch();
    if (!Lp) return fail(KIN_ENOMEM, "host allocation failed");
    struct Free { Launch* p; ~Free() { delete p; } } fr{Lp};
    Launch& P = *Lp;
    int64_t total = 0;
    for (int i = 0; i < n; ++i) {
        const kin_instance& I = inst[i];
        if (I.cells < 0) return fail(KIN_EINVAL, "instance %d: cells < 0", i);
        if (!finite_pos(I.dt)) return fail(KIN_EINVAL, "instance %d: dt must be finite and > 0", i);
        if (!finite_pos(I.rtol)) return fail(KIN_EINVAL, "instance %d: rtol must be finite and > 0", i);
        if (!std::isfinite(I.atol) || I.atol < 0) return fail(KIN_EINVAL, "instance %d: atol must be finite and >= 0", i);
        if (I.cells > 0) {
            if (!I.T || !I.p || !I.Y) return fail(KIN_EINVAL, "instance %d: T, p and Y must be non-NULL", i);
            if (I.ldY < I.cells) return fail(KIN_EINVAL, "instance %d: ldY < cells", i);
            if (I.ldY > INT32_MAX) return fail(KIN_EINVAL, "instance %d: ldY >= 2^31", i);
            if (!is_device_ptr(I.T) || !is_device_ptr(I.p) || !is_device_ptr(I.Y) ||
                (I.status && !is_device_ptr(I.status)) || (I.stats && !is_device_ptr(I.stats)))
                return fail(KIN_EINVAL, "instance %d: T, p, Y, status and stats must be device memory", i);
        }
        P.start[i] = total;
        P.inst[i] = InstDev{I.T, I.p, I.Y, I.ldY, I.dt, I.rtol, I.atol, I.status, I.stats};
        total += I.cells;
    }
    P.start[n] = total;
    if (total == 0) return KIN_OK;
    Grid g;
    rc = grid_for(m, o, total, &g);
    if (rc) return rc;
    const int64_t need = ws_bytes(m, o, g, total);
    if (!ws) return fail(KIN_EINVAL, "workspace is NULL");
    if (((uintptr_t)ws) % 256) return fail(KIN_EINVAL, "workspace must be 256-byte aligned");
    if (ws_size < need) return fail(KIN_ENOMEM, "workspace has %lld bytes, needs %lld", (long long)ws_size, (long long)need);
    if (!is_device_ptr(ws)) return fail(KIN_EINVAL, "workspace must be device memory");
    // never more lanes (warps in the warp layout) than cells
    int blocks = g.blocks;
    const int per_block = g.layout == KIN_LAYOUT_WARP
                              ? g.threads / warp_cell_lanes(o->method, m->nS + o->energy)
                              : g.threads;
    const int64_t want = (total + per_block - 1) / per_block;
    if (want < blocks) blocks = (int)want;
    const int64_t nslots = (int64_t)blocks * g.threads;
    P.M = m->dev;
    P.method = o->method;
    P.precision = o->precision;
    P.max_steps = o->max_steps > 0 ? o->max_steps : 100000;
    P.n_inst = n;
    P.nslots = nslots;
    P.total = total;
    char* base = (char*)ws;
    const int sig = o->method == KIN_RKC ? o->sigma : KIN_SIGMA_GERSHGORIN;
    const WsLayout w = ws_layout(m->dev, o->precision, sig, o->energy,
                                 g.layout == KIN_LAYOUT_WARP ? 0 : nslots, total);
    P.energy = o->energy;
    P.nV = m->nS + o->energy;
    P.sigma_method = sig;
    P.cell_ev = sig == KIN_SIGMA_POWER ? (double*)(base + w.ev) : nullptr;
    P.queue = (unsigned long long*)(base + w.header);
    P.hist = (unsigned*)(base + w.header + 256);
    P.vec = (double*)(base + w.vec);
    P.lane_r = base + w.lane_r;
    P.lane_sig = (double*)(base + w.lane_sig);
    P.cell_k = base + w.cell_k;
    P.cell_f0 = (double*)(base + w.f0);
    P.cell_sig = (double*)(base + w.sig);
    P.cell_h = (double*)(base + w.h);
    P.cell_nfe = (int32_t*)(base + w.nfe);
    P.cell_nfs = (int32_t*)(base + w.nfs);
    P.cell_st = (uint8_t*)(base + w.st);
    P.order = (int32_t*)(base + w.order);
    if (total > INT32_MAX) return fail(KIN_EINVAL, "more than 2^31-1 cells in one call");
    // f: tables, or the mechanism's generated code (lane layout, FP64, isothermal)
    bool gen = false;
    GenKernels gk{};
    // (the automatic choice leaves the energy equation on the tables: with a
    // per-reaction exp inlined, the generated form measured slower)
    if (o->feval == KIN_FEVAL_GENERATED ||
        (o->feval == KIN_FEVAL_AUTO && total >= KIN_GEN_MIN_CELLS && !o->energy)) {
        // (the energy equation comes generated too: the mechanism has cp and
        // Hf, checked above, so its source carries that form of f)
        const bool serves = g.layout == KIN_LAYOUT_LANE && o->precision == KIN_FP64 &&
                            o->staging == KIN_STAGE_GLOBAL && !m->gen_src.empty();
        if (serves) {
            std::string log;
            const int grc = gen_kernels(m->device, m->gen_src, &gk, &log);
            if (grc == KIN_OK && (!o->energy || gk.energy)) gen = true;
            else if (o->feval == KIN_FEVAL_GENERATED)
                return fail(grc != KIN_OK ? grc : KIN_EUNSUPPORTED, "generated f: %.400s", log.c_str());
        } else if (o->feval == KIN_FEVAL_GENERATED) {
            return fail(KIN_EUNSUPPORTED, "the generated f serves the lane layout, KIN_FP64, "
                                          "KIN_STAGE_GLOBAL and at most %d species / %d reactions",
                        KIN_GEN_MAX_SPECIES, KIN_GEN_MAX_REACTIONS);
        }
    }
    cudaStream_t st = (cudaStream_t)o->stream;
    cudaError_t e = cudaMemsetAsync(base + w.header, 0, 512, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    if (g.layout == KIN_LAYOUT_WARP && o->method == KIN_RKCK) {
        e = o->precision == KIN_MIXED ? launch_warp_rkck_f32(P, blocks, g.threads, st)
                                      : launch_warp_rkck_f64(P, blocks, g.threads, st);
    } else if (g.layout == KIN_LAYOUT_WARP) {
        using LaunchFn = cudaError_t (*)(Launch&, int, int, cudaStream_t);
        // [energy][precision][occupancy]
        static const LaunchFn fns[2][2][2] = {
            {{launch_warp_f64_o0, launch_warp_f64_o1}, {launch_warp_f32_o0, launch_warp_f32_o1}},
            {{launch_warp_f64_en_o0, launch_warp_f64_en_o1}, {launch_warp_f32_en_o0, launch_warp_f32_en_o1}}};
        e = fns[o->energy][o->precision == KIN_MIXED][o->occupancy ? 1 : 0](P, blocks, g.threads, st);
    }
    else if (gen)
        e = gen_launch(gk, P, o->occupancy, blocks, g.threads, st);
    else
        e = launch_integrate(P, o->energy ? KIN_STAGE_GLOBAL : o->staging, o->occupancy, blocks,
                             g.threads, st);
    if (e != cudaSuccess) return cuda_fail(e, "integrate launch");
    return KIN_OK;
}

int kin_integrate(const kin_mech* m, int64_t cells, double* T, const double* p, double* Y,
                  int64_t ldY, double dt, double rtol, double atol, const kin_opts* o,
                  uint8_t* status, int32_t* stats, void* ws, int64_t ws_size)
{
    kin_instance I{cells, T, p, Y, ldY, dt, rtol, atol, status, stats};
    return kin_integrate_batch(m, 1, &I, o, ws, ws_size);
}

static int64_t al256(int64_t x) { return (x + 255) / 256 * 256; }

int64_t kin_host_buffer_bytes(const kin_mech* m, const kin_opts* o, int64_t cells)
{
    g_err[0] = 0;
    if (cells < 0) return fail(KIN_EINVAL, "cells < 0");
    int64_t ws = kin_workspace_bytes(m, o, cells);
    if (ws < 0) return ws;
    return al256(ws) + 2 * al256(8 * cells) + al256(8 * cells * m->nS) + al256(cells) + al256(4 * KIN_NSTATS * cells);
}

int kin_integrate_host(const kin_mech* m, int64_t cells, double* T, const double* p, double* Y,
                       int64_t ldY, double dt, double rtol, double atol, const kin_opts* o,
                       uint8_t* status, int32_t* stats, void* buf, int64_t bytes)
{
    g_err[0] = 0;
    const int64_t need = kin_host_buffer_bytes(m, o, cells);
    if (need < 0) return (int)need;
    if (cells == 0) return KIN_OK;
    if (!T || !p || !Y) return fail(KIN_EINVAL, "T, p and Y must be non-NULL");
    if (ldY < cells) return fail(KIN_EINVAL, "ldY < cells");
    if (!buf || ((uintptr_t)buf) % 256) return fail(KIN_EINVAL, "device_buffer must be non-NULL and 256-byte aligned");
    if (bytes < need) return fail(KIN_ENOMEM, "device_buffer has %lld bytes, needs %lld", (long long)bytes, (long long)need);
    if (!is_device_ptr(buf)) return fail(KIN_EINVAL, "device_buffer must be device memory");
    const int64_t ws = kin_workspace_bytes(m, o, cells);
    char* b = (char*)buf;
    int64_t off = al256(ws);
    double* Td = (double*)(b + off); off += al256(8 * cells);
    double* pd = (double*)(b + off); off += al256(8 * cells);
    double* Yd = (double*)(b + off); off += al256(8 * cells * m->nS);
    uint8_t* sd = (uint8_t*)(b + off); off += al256(cells);
    int32_t* xd = (int32_t*)(b + off);
    cudaStream_t st = (cudaStream_t)o->stream;
    cudaError_t e = cudaMemcpyAsync(Td, T, 8 * cells, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(pd, p, 8 * cells, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(Yd, 8 * cells, Y, 8 * ldY, 8 * cells, m->nS, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "host-to-device copy");
    int rc = kin_integrate(m, cells, Td, pd, Yd, cells, dt, rtol, atol, o, sd, stats ? xd : nullptr, buf, ws);
    if (rc) return rc;
    e = cudaMemcpy2DAsync(Y, 8 * ldY, Yd, 8 * cells, 8 * cells, m->nS, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && o->energy) e = cudaMemcpyAsync(T, Td, 8 * cells, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && status) e = cudaMemcpyAsync(status, sd, cells, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && stats) e = cudaMemcpyAsync(stats, xd, 4 * KIN_NSTATS * cells, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(e, "device-to-host copy");
    return KIN_OK;
}

int kin_rates(const kin_mech* m, int64_t cells, const double* T, const double* p, const double* Y,
              int64_t ldY, double* dYdt, int32_t precision, void* stream, void* ws, int64_t ws_size)
{
    g_err[0] = 0;
    if (!m) return fail(KIN_EINVAL, "mechanism is NULL");
    if (precision != KIN_FP64 && precision != KIN_MIXED) return fail(KIN_EINVAL, "unknown precision %d", precision);
    if (cells < 0) return fail(KIN_EINVAL, "cells < 0");
    if (cells == 0) return KIN_OK;
    if (!T || !p || !Y || !dYdt) return fail(KIN_EINVAL, "T, p, Y and dYdt must be non-NULL");
    if (ldY < cells) return fail(KIN_EINVAL, "ldY < cells");
    if (ldY > INT32_MAX) return fail(KIN_EINVAL, "ldY >= 2^31");
    if (!is_device_ptr(T) || !is_device_ptr(p) || !is_device_ptr(Y) || !is_device_ptr(dYdt))
        return fail(KIN_EINVAL, "T, p, Y and dYdt must be device memory");
    kin_opts o{KIN_RKC, precision, 0, 0, 0, KIN_STAGE_GLOBAL, KIN_OCC_DEFAULT, 0, KIN_LAYOUT_LANE, 0,
               KIN_FEVAL_TABLE, stream};
    Grid g;
    int rc = grid_for(m, &o, cells, &g);
    if (rc) return rc;
    const int64_t need = ws_bytes(m, &o, g, cells);
    if (!ws || ((uintptr_t)ws) % 256) return fail(KIN_EINVAL, "workspace must be non-NULL and 256-byte aligned");
    if (ws_size < need) return fail(KIN_ENOMEM, "workspace has %lld bytes, needs %lld", (long long)ws_size, (long long)need);
    if (!is_device_ptr(ws)) return fail(KIN_EINVAL, "workspace must be device memory");
    cudaError_t e = launch_rates(m->dev, cells, T, p, Y, ldY, dYdt, precision, ws, g.nslots,
                                 g.blocks, g.threads, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "rates launch");
    return KIN_OK;
}

}  // extern "C"
