// kin_dev.cuh -- device-side data layout shared by the kernels and the host ABI.
//
// Mechanism tables live in one device allocation owned by kin_mech. Per-lane
// working arrays live in the caller's workspace, laid out element-major
// ([element][lane]) so that the 32 lanes of a warp touching element e of
// their own cells hit 32 consecutive words (coalesced), whatever the
// mechanism size.
#pragma once
#include <cstdint>

#include "../../include/kin.h"

namespace kin {

constexpr double R_GAS = 8.314462618;  // J/(mol K)
constexpr int SMAX = KIN_MAX_STAGES;
constexpr int RKC_TAB_S = SMAX + 1;    // rows s = 0..250 (2..250 used)
constexpr int RKC_TAB_W = 5;           // mu, nu, mu~, gamma~, 1 - mu - nu

// Per-reaction descriptor: reactant slots, type, efficiency row.
struct Rxn {
    int r0, r1;  // reactant species or -1
    int type;    // KIN_RXN_*
    int row;     // efficiency row or -1
};

struct MechDev {
    int nS, nR, nM, nnz;
    const double* W;       // [nS]
    const double* invW;    // [nS]
    const float* invW32;   // [nS]
    const double* lnA;     // [nR]
    const double* beta;    // [nR]
    const double* EaR;     // [nR] Ea / R (K)
    const double* lnA0;    // [nR]
    const double* beta0;   // [nR]
    const double* Ea0R;    // [nR]
    const Rxn* rxn;        // [nR]
    const int* csr_ptr;    // [nS + 1] species -> entries
    const int* csr_rxn;    // [nnz] reaction of each entry (ascending per species)
    const double* csr_nu;  // [nnz] net coefficient nu'' - nu' of the species
    const float* csr_nu32; // [nnz]
    const double* eff;     // [nM][nS]
    const float* eff32;    // [nM][nS]
    const double* rkc;     // [RKC_TAB_S][RKC_TAB_S][RKC_TAB_W]
};

// One instance of a batched launch (device pointers).
struct InstDev {
    const double* T;
    const double* p;
    double* Y;
    int64_t ldY;
    double dt, rtol, atol;
    uint8_t* status;
    int32_t* stats;
};

// Number of FP64 working vectors of nS entries each, per lane.
constexpr int NVEC = 8;

struct Launch {
    MechDev M;
    int method, precision, max_steps, n_inst;
    int64_t nslots;                 // lanes in the persistent grid
    unsigned long long* queue;      // next global cell index
    double* vec;                    // [NVEC * nS][nslots]
    void* rarr;                     // [2 nR + nS + nR][nslots] of the rate type
    int64_t total;                  // cells over all instances
    int64_t start[KIN_MAX_INSTANCES + 1];  // prefix sums of instance cells
    InstDev inst[KIN_MAX_INSTANCES];
};

// Host-side helpers implemented in kernels.cu.
int64_t scratch_elems_vec(int nS);
int64_t scratch_bytes_rate(int nS, int nR, int precision);
cudaError_t launch_integrate(const Launch& L, int blocks, int threads, cudaStream_t st);
cudaError_t launch_rates(const MechDev& M, int64_t cells, const double* T, const double* p,
                         const double* Y, int64_t ldY, double* dYdt, int precision,
                         void* rarr, int64_t nslots, int blocks, int threads, cudaStream_t st);
cudaError_t launch_rkc_table(double* tab, cudaStream_t st);
cudaError_t integrate_occupancy(int method, int precision, int threads, int* blocks_per_sm);

}  // namespace kin
