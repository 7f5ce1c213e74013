// kin_dev.cuh -- device-side data layout shared by the kernels and the host ABI.
//
// Mechanism tables live in one device allocation owned by kin_mech. Working
// arrays live in the caller's workspace, laid out element-major
// ([element][lane] or [element][cell]) so that the 32 lanes of a warp touching
// element e of their own cells hit consecutive words.
#pragma once
#ifndef __CUDACC_RTC__
#include <cstdint>
#endif

#include "../../include/kin.h"

namespace kin {

constexpr double R_GAS = 8.314462618;  // J/(mol K)
constexpr double T_REF = 298.15;        // K, reference of the formation enthalpies
constexpr int SMAX = KIN_MAX_STAGES;
constexpr int RKC_TAB_S = SMAX + 1;    // rows s = 0..250 (2..250 used)
constexpr int RKC_TAB_W = 5;           // mu, nu, mu~, gamma~, 1 - mu - nu
constexpr int NBUCKET = 64;            // cost buckets of the longest-first order

// Per-reaction descriptor (16 bytes).
struct Rxn {
    int16_t r0, r1;  // reactant species or -1
    int16_t type;    // KIN_RXN_*
    int16_t pad;
    int32_t row;     // efficiency row or -1
    int32_t fo;      // falloff ordinal or -1
};

// Stoichiometric entry of the warp layout's gather: the net coefficient
// times the species' molar mass, and the reaction's permutation position.
struct CsrW32 {
    float nuW;
    int32_t pos;
};
struct CsrW64 {
    double nuW;
    int32_t pos, pad;
};

// Species slots of 32 in the warp layout's ELL gather tables.
constexpr int ELL_SLOTS = (KIN_MAX_SPECIES + 31) / 32;

struct MechDev {
    int nS, nR, nM, nFO, nnz;
    const double* W;       // [nS]
    const float* W32;      // [nS]
    const double* invW;    // [nS]
    const float* invW32;   // [nS]
    const double* lnA;     // [nR]
    const double* beta;    // [nR]
    const double* EaR;     // [nR] Ea / R (K)
    const double* lnA0;    // [nR]
    const double* beta0;   // [nR]
    const double* Ea0R;    // [nR]
    const Rxn* rxn;        // [nR]
    // warp-per-cell layout: reactions in the order plain, third-body, falloff
    const int* rxn_perm;   // [nR] reaction at each permutation position
    const Rxn* rxnp;       // [nR] descriptors in permutation order; .row indexes effT's columns
    const int* csrp_rxn;   // [nnz] permutation position of each CSR entry's reaction
    // The same entries for a 32-lane gather, in ELL order: species i = 32 r + l
    // keeps its k-th entry at ell[ell_base[r] + 32 k + l] (k below the row
    // length csr_ptr[i + 1] - csr_ptr[i]), so the 32 lanes of a step read
    // consecutive entries.
    const CsrW32* ell32;
    const CsrW64* ell64;
    int ell_base[ELL_SLOTS];
    // The segmented FP32 gather of the 32-lane isothermal f (seg_tables.h):
    // the nonzeros cut into 32 equal chunks of seg_K packed entries, one per
    // lane. Null where the packed form does not apply (the ELL gather runs).
    const uint32_t* seg_ent;   // [seg_K][32] nu's FP32 bits | flush flag | position
    const int32_t* seg_slot0;  // [32] first partial slot of each lane
    const int32_t* seg_part;   // [nS] first slot << 8 | slot count; -1: empty row
    int seg_K;
    // efficiencies by non-plain reaction in permutation order (row), species
    // in 16-byte groups: [k / V][row][k % V], V = 2 (FP64) or 4 (FP32), the
    // last group zero-padded
    const double* effV64;
    const float* effV32;
    // reactants of each reaction in permutation order: (r0 + 1) | (r1 + 1) << 16
    const uint32_t* rxw;
    const int* csr_ptr;    // [nS + 1] species -> entries
    const int* csr_rxn;    // [nnz] reaction of each entry (ascending per species)
    const double* csr_nu;  // [nnz] net coefficient nu'' - nu' of the species
    const float* csr_nu32; // [nnz]
    const double* csr_nuW; // [nnz] nu'' - nu' times the species' W (isothermal f: dY/dt = (sum) / rho)
    const float* csr_nuW32; // [nnz]
    const double* eff;     // [nM][nS]
    const float* eff32;    // [nM][nS]
    const double* rkc;     // [RKC_TAB_S][RKC_TAB_S][RKC_TAB_W]
    // energy equation (null without thermochemistry)
    const double* cp;      // [nS] J/(mol K)
    const double* cpW;     // [nS] cp_i / W_i, J/(g K)
    const double* Hf;      // [nS] J/mol at T_REF
};

// One instance of a batched launch (device pointers).
struct InstDev {
    double* T;  // written back with the energy equation
    const double* p;
    double* Y;
    int64_t ldY;
    double dt, rtol, atol;
    uint8_t* status;
    int32_t* stats;
};

// FP64 working vectors of nS entries per lane.
constexpr int NVEC = 8;

struct Launch {
    MechDev M;
    int method, precision, max_steps, n_inst, sigma_method;
    int energy;  // 1: T is state component nS (Eq. (E:energy))
    int nV;      // state length: nS + energy
    int64_t nslots;                 // lanes of the persistent grid
    int64_t total;                  // cells over all instances
    unsigned long long* queue;      // next position in `order`
    unsigned* hist;                 // [NBUCKET] counts, then cursors
    // per lane
    double* vec;                    // [NVEC * nV][nslots]
    void* lane_r;                   // C [nS], Omega [nR], k [nR], k0/kinf [nFO] of the rate
                                    // type: [nS + 2 nR + nFO][nslots]
    double* lane_sig;               // mixed precision: FP64 C [nS], Omega [nR] for the
                                    // spectral-radius evaluations of f: [nS + nR][nslots]
    // per cell (global cell index g over all instances)
    void* cell_k;                   // k_j [nR][total], then k0/kinf [nFO][total], rate type
    double* cell_f0;                // f(y0) [nV][total]
    double* cell_ev;                // power-method direction [nV][total] (power sigma only)
    double* cell_sig;               // RKC spectral radius at y0 [total]
    double* cell_h;                 // first trial step [total]
    int32_t* cell_nfe;              // f evaluations spent before the main kernel [total]
    int32_t* cell_nfs;              // ... of which inside the spectral-radius estimate [total]
    uint8_t* cell_st;               // 0, or a final status decided before the main kernel
    int32_t* order;                 // processing order (longest predicted first) [total]
    int64_t start[KIN_MAX_INSTANCES + 1];  // prefix sums of instance cells
    InstDev inst[KIN_MAX_INSTANCES];
};

// Workspace layout for `cells` cells and `nslots` lanes.
struct WsLayout {
    int64_t header, vec, lane_r, lane_sig, cell_k, f0, ev, sig, h, nfe, nfs, st, order, total;
};
WsLayout ws_layout(const MechDev& M, int precision, int sigma_method, int energy, int64_t nslots,
                   int64_t cells);

#ifndef __CUDACC_RTC__  // host-side declarations (absent from run-time compiled code)
// Host-side helpers implemented in kernels.cu.
cudaError_t launch_integrate(Launch& L, int staging, int occupancy, int blocks, int threads,
                             cudaStream_t st);
size_t smem_bytes(const MechDev& M, int precision, int threads, int staging);
cudaError_t launch_rates(const MechDev& M, int64_t cells, const double* T, const double* p,
                         const double* Y, int64_t ldY, double* dYdt, int precision, void* ws,
                         int64_t nslots, int blocks, int threads, cudaStream_t st);
cudaError_t launch_rkc_table(double* tab, cudaStream_t st);
// Per method/precision instantiations (inst_*.cu) and the bucket sort.
cudaError_t launch_rkc_f64(Launch& L, int stg, int occ, int blocks, int threads, cudaStream_t st);
cudaError_t launch_rkc_f32(Launch& L, int stg, int occ, int blocks, int threads, cudaStream_t st);
cudaError_t launch_rkck_f64(Launch& L, int stg, int occ, int blocks, int threads, cudaStream_t st);
cudaError_t launch_rkck_f32(Launch& L, int stg, int occ, int blocks, int threads, cudaStream_t st);
cudaError_t occ_rkc_f64(int stg, int occ, int threads, size_t sm, int* bps);
cudaError_t occ_rkc_f32(int stg, int occ, int threads, size_t sm, int* bps);
cudaError_t occ_rkck_f64(int stg, int occ, int threads, size_t sm, int* bps);
cudaError_t occ_rkck_f32(int stg, int occ, int threads, size_t sm, int* bps);
cudaError_t launch_sort(Launch& L, cudaStream_t st);
// Energy-equation variants of the lane kernels (inst_energy_*.cu, staging 0).
cudaError_t launch_rkc_f64_en(Launch& L, int occ, int blocks, int threads, cudaStream_t st);
cudaError_t launch_rkc_f32_en(Launch& L, int occ, int blocks, int threads, cudaStream_t st);
cudaError_t launch_rkck_f64_en(Launch& L, int occ, int blocks, int threads, cudaStream_t st);
cudaError_t launch_rkck_f32_en(Launch& L, int occ, int blocks, int threads, cudaStream_t st);
cudaError_t occ_rkc_f64_en(int occ, int threads, size_t sm, int* bps);
cudaError_t occ_rkc_f32_en(int occ, int threads, size_t sm, int* bps);
cudaError_t occ_rkck_f64_en(int occ, int threads, size_t sm, int* bps);
cudaError_t occ_rkck_f32_en(int occ, int threads, size_t sm, int* bps);
// Warp-per-cell RKC (inst_warp_*.cu): one warp integrates one cell; one
// translation unit per rate precision and register budget (occupancy).
cudaError_t launch_warp_f64_o0(Launch& L, int blocks, int threads, cudaStream_t st);
cudaError_t launch_warp_f64_o1(Launch& L, int blocks, int threads, cudaStream_t st);
cudaError_t launch_warp_f32_o0(Launch& L, int blocks, int threads, cudaStream_t st);
cudaError_t launch_warp_f32_o1(Launch& L, int blocks, int threads, cudaStream_t st);
cudaError_t occ_warp_f64_o0(const MechDev& M, int nV, int threads, int* bps);
cudaError_t occ_warp_f64_o1(const MechDev& M, int nV, int threads, int* bps);
cudaError_t occ_warp_f32_o0(const MechDev& M, int nV, int threads, int* bps);
cudaError_t occ_warp_f32_o1(const MechDev& M, int nV, int threads, int* bps);
cudaError_t launch_warp_f64_en_o0(Launch& L, int blocks, int threads, cudaStream_t st);
cudaError_t launch_warp_f64_en_o1(Launch& L, int blocks, int threads, cudaStream_t st);
cudaError_t launch_warp_f32_en_o0(Launch& L, int blocks, int threads, cudaStream_t st);
cudaError_t launch_warp_f32_en_o1(Launch& L, int blocks, int threads, cudaStream_t st);
cudaError_t occ_warp_f64_en_o0(const MechDev& M, int nV, int threads, int* bps);
cudaError_t occ_warp_f64_en_o1(const MechDev& M, int nV, int threads, int* bps);
cudaError_t occ_warp_f32_en_o0(const MechDev& M, int nV, int threads, int* bps);
cudaError_t occ_warp_f32_en_o1(const MechDev& M, int nV, int threads, int* bps);
cudaError_t launch_warp_rkck_f64(Launch& L, int blocks, int threads, cudaStream_t st);
cudaError_t launch_warp_rkck_f32(Launch& L, int blocks, int threads, cudaStream_t st);
cudaError_t occ_warp_rkck_f64(const MechDev& M, int nV, int energy, int threads, int* bps);
cudaError_t occ_warp_rkck_f32(const MechDev& M, int nV, int energy, int threads, int* bps);
// Dynamic shared memory of a 32-lane warp's worth of cell groups per block of
// `threads` (RKC: one cell per warp; RKCK with 16-lane groups: multiply by 2).
size_t warp_smem(const MechDev& M, int precision, int energy, int threads);

// Lanes that integrate one cell in the warp-per-cell layout: a whole warp,
// or half of one (two cells per warp) for RKCK on states of at most 16
// components.
inline int warp_cell_lanes(int method, int nV) { return method == KIN_RKCK && nV <= 16 ? 16 : 32; }

// Record `code` and a printf-style message as the calling thread's last
// error (kin_last_error); returns `code`.
int set_last_error(int code, const char* fmt, ...);
// Options under which a call of `cells` cells runs in a fixed working array of
// `cap_bytes` without allocating (abi.cu): the f evaluation never compiles
// (the generated f only where it is already loaded on the device), and the
// requested blocks per SM (0: as many as fit) step down to the largest count
// whose workspace fits. KIN_ENOMEM if none fits; other errors as
// kin_workspace_bytes.
int noalloc_opts(const kin_mech* m, const kin_opts* in, int64_t cells, int64_t cap_bytes,
                 kin_opts* out);
cudaError_t integrate_occupancy(const MechDev& M, int method, int precision, int staging,
                                int occupancy, int energy, int threads, int* blocks_per_sm);
#endif  // __CUDACC_RTC__

}  // namespace kin
