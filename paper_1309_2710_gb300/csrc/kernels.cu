// kernels.cu -- non-template kernels and host launchers of the integrator:
// the f-alone kernel, the RKC coefficient table, the longest-first bucket
// sort, workspace layout, and dispatch to the per-method/precision
// instantiations (inst_*.cu).
#include "kernels.cuh"

namespace kin {

__global__ void bucket_count_kernel(const __grid_constant__ Launch L)
{
    __shared__ unsigned h[NBUCKET];
    for (int i = threadIdx.x; i < NBUCKET; i += blockDim.x) h[i] = 0;
    __syncthreads();
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < L.total;
         g += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&h[cost_bucket(L, g)], 1u);
    __syncthreads();
    for (int i = threadIdx.x; i < NBUCKET; i += blockDim.x)
        if (h[i]) atomicAdd(&L.hist[i], h[i]);
}

// Exclusive scan in descending bucket order: the costliest bucket first.
__global__ void bucket_scan_kernel(unsigned* hist)
{
    if (threadIdx.x == 0) {
        unsigned run = 0;
        for (int b = NBUCKET - 1; b >= 0; --b) {
            const unsigned n = hist[b];
            hist[b] = run;
            run += n;
        }
    }
}

__global__ void bucket_scatter_kernel(const __grid_constant__ Launch L)
{
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < L.total;
         g += (int64_t)gridDim.x * blockDim.x) {
        const unsigned pos = atomicAdd(&L.hist[cost_bucket(L, g)], 1u);
        L.order[pos] = (int32_t)g;
    }
}

// ------------------------------------------------------------- f alone ---
template <typename R>
__global__ void rates_kernel(MechDev M, int64_t cells, const double* __restrict__ T,
                             const double* __restrict__ p, const double* Y, int64_t ldY,
                             double* dYdt, void* lane_r, void* cell_k, int64_t nslots)
{
    const int64_t slot = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (slot >= nslots) return;
    R* rb = reinterpret_cast<R*>(lane_r) + slot;
    Lane<R> C{rb, (int32_t)nslots}, OM{rb + (int64_t)M.nS * nslots, (int32_t)nslots};
    for (int64_t c = slot; c < cells; c += nslots) {
        Lane<R> K{reinterpret_cast<R*>(cell_k) + c, (int32_t)cells};
        Lane<R> KR{reinterpret_cast<R*>(cell_k) + (int64_t)M.nR * cells + c, (int32_t)cells};
        rate_constants<R>(M, T[c], K, KR);
        const double Ctot = p[c] * 1e-6 / (R_GAS * T[c]);
        feval<R>(M, Ctot, 1.0 / Ctot, K, KR, C, OM,
                 Lane<double>{const_cast<double*>(Y) + c, (int32_t)ldY}, Lane<double>{dYdt + c, (int32_t)ldY});
    }
}

// ------------------------------------------------ RKC coefficient table ---
// Section 2.3: w0 = 1 + kappa/s^2 (kappa = 2/13), Chebyshev T_j, T_j', T_j''
// at w0 by the three-term recursion, b_j = T_j''/T_j'^2 (b_0 = b_1 = b_2),
// a_j = 1 - b_j T_j(w0), w1 = T_s'/T_s'', mu~_1 = b_1 w1 and for j >= 2
// mu_j = 2 b_j w0/b_{j-1}, nu_j = -b_j/b_{j-2}, mu~_j = 2 b_j w1/b_{j-1},
// gamma~_j = -a_{j-1} mu~_j. One thread per stage count s.
__global__ void rkc_table_kernel(double* tab)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < 2 || s > SMAX) return;
    const double w0 = 1.0 + (2.0 / 13.0) / ((double)s * s);
    double t0 = 1.0, t1 = w0, d0 = 0.0, d1 = 1.0, e0 = 0.0, e1 = 0.0;
    for (int j = 2; j <= s; ++j) {
        const double t2 = 2.0 * w0 * t1 - t0;
        const double d2 = 2.0 * t1 + 2.0 * w0 * d1 - d0;
        const double e2 = 4.0 * d1 + 2.0 * w0 * e1 - e0;
        t0 = t1; t1 = t2; d0 = d1; d1 = d2; e0 = e1; e1 = e2;
    }
    const double w1 = d1 / e1;
    t0 = 1.0; t1 = w0; d0 = 0.0; d1 = 1.0; e0 = 0.0; e1 = 0.0;
    const double b2 = 4.0 / (16.0 * w0 * w0);  // T_2''/T_2'^2 = 4 / (4 w0)^2
    double bjm2 = b2, bjm1 = b2;                // b_0, b_1
    double ajm1 = 1.0 - b2 * w0;                // a_1 = 1 - b_1 T_1(w0)
    double* row1 = tab + ((int64_t)s * RKC_TAB_S + 1) * RKC_TAB_W;
    row1[0] = row1[1] = row1[3] = row1[4] = 0.0;
    row1[2] = b2 * w1;
    for (int j = 2; j <= s; ++j) {
        const double t2 = 2.0 * w0 * t1 - t0;
        const double d2 = 2.0 * t1 + 2.0 * w0 * d1 - d0;
        const double e2 = 4.0 * d1 + 2.0 * w0 * e1 - e0;
        const double bj = e2 / (d2 * d2);
        const double mu = 2.0 * bj * w0 / bjm1;
        const double nu = -bj / bjm2;
        const double mt = 2.0 * bj * w1 / bjm1;
        const double gt = -ajm1 * mt;
        double* r = tab + ((int64_t)s * RKC_TAB_S + j) * RKC_TAB_W;
        r[0] = mu;
        r[1] = nu;
        r[2] = mt;
        r[3] = gt;
        r[4] = 1.0 - mu - nu;
        ajm1 = 1.0 - bj * t2;
        bjm2 = bjm1;
        bjm1 = bj;
        t0 = t1; t1 = t2; d0 = d1; d1 = d2; e0 = e1; e1 = e2;
    }
}

// -------------------------------------------------------- host launchers --
static int64_t al256(int64_t x) { return (x + 255) / 256 * 256; }

WsLayout ws_layout(const MechDev& M, int precision, int sigma_method, int energy, int64_t nslots,
                   int64_t cells)
{
    const int64_t rb = precision == KIN_MIXED ? 4 : 8;
    const int64_t nV = M.nS + (energy ? 1 : 0);
    WsLayout w;
    int64_t off = 0;
    w.header = off;  off += 4096;
    w.vec = off;     off += al256((int64_t)NVEC * nV * 8 * nslots);
    w.lane_r = off;  off += al256((int64_t)(M.nS + 2 * M.nR + M.nFO) * rb * nslots);
    w.lane_sig = off; off += precision == KIN_MIXED ? al256((int64_t)(M.nS + M.nR) * 8 * nslots) : 0;
    // rate constants per cell, unless they follow T (energy equation)
    w.cell_k = off;  off += energy ? 0 : al256((int64_t)(M.nR + M.nFO) * rb * cells);
    w.f0 = off;      off += al256(nV * 8 * cells);
    w.ev = off;      off += sigma_method == KIN_SIGMA_POWER ? al256(nV * 8 * cells) : 0;
    w.sig = off;     off += al256(8 * cells);
    w.h = off;       off += al256(8 * cells);
    w.nfe = off;     off += al256(4 * cells);
    w.nfs = off;     off += al256(4 * cells);
    w.st = off;      off += al256(cells);
    w.order = off;   off += al256(4 * cells);
    w.total = off;
    return w;
}

size_t smem_bytes(const MechDev& M, int precision, int threads, int stg)
{
    const size_t n = (stg >= 1 ? M.nS + M.nR : 0) + (stg >= 2 ? M.nR + M.nFO : 0);
    return n * threads * (precision == KIN_MIXED ? 4 : 8);
}

cudaError_t launch_integrate(Launch& L, int stg, int occ, int blocks, int threads, cudaStream_t st)
{
    if (L.energy) {
        if (L.method == KIN_RKCK)
            return L.precision == KIN_MIXED ? launch_rkck_f32_en(L, occ, blocks, threads, st)
                                            : launch_rkck_f64_en(L, occ, blocks, threads, st);
        return L.precision == KIN_MIXED ? launch_rkc_f32_en(L, occ, blocks, threads, st)
                                        : launch_rkc_f64_en(L, occ, blocks, threads, st);
    }
    if (L.method == KIN_RKCK)
        return L.precision == KIN_MIXED ? launch_rkck_f32(L, stg, occ, blocks, threads, st)
                                        : launch_rkck_f64(L, stg, occ, blocks, threads, st);
    return L.precision == KIN_MIXED ? launch_rkc_f32(L, stg, occ, blocks, threads, st)
                                    : launch_rkc_f64(L, stg, occ, blocks, threads, st);
}

cudaError_t integrate_occupancy(const MechDev& M, int method, int precision, int stg, int occ,
                                int energy, int threads, int* bps)
{
    if (energy) {
        if (method == KIN_RKCK)
            return precision == KIN_MIXED ? occ_rkck_f32_en(occ, threads, 0, bps)
                                          : occ_rkck_f64_en(occ, threads, 0, bps);
        return precision == KIN_MIXED ? occ_rkc_f32_en(occ, threads, 0, bps)
                                      : occ_rkc_f64_en(occ, threads, 0, bps);
    }
    const size_t sm = smem_bytes(M, precision, threads, stg);
    if (method == KIN_RKCK)
        return precision == KIN_MIXED ? occ_rkck_f32(stg, occ, threads, sm, bps)
                                      : occ_rkck_f64(stg, occ, threads, sm, bps);
    return precision == KIN_MIXED ? occ_rkc_f32(stg, occ, threads, sm, bps)
                                  : occ_rkc_f64(stg, occ, threads, sm, bps);
}

cudaError_t launch_sort(Launch& L, cudaStream_t st)
{
    const int64_t nb = (L.total + 255) / 256;
    const int sb = (int)(nb < 1024 ? nb : 1024);
    bucket_count_kernel<<<sb, 256, 0, st>>>(L);
    bucket_scan_kernel<<<1, 32, 0, st>>>(L.hist);
    bucket_scatter_kernel<<<sb, 256, 0, st>>>(L);
    return cudaGetLastError();
}

cudaError_t launch_rates(const MechDev& M, int64_t cells, const double* T, const double* p,
                         const double* Y, int64_t ldY, double* dYdt, int precision, void* ws,
                         int64_t nslots, int blocks, int threads, cudaStream_t st)
{
    const WsLayout w = ws_layout(M, precision, KIN_SIGMA_GERSHGORIN, 0, nslots, cells);
    char* b = (char*)ws;
    if (precision == KIN_MIXED)
        rates_kernel<float><<<blocks, threads, 0, st>>>(M, cells, T, p, Y, ldY, dYdt, b + w.lane_r,
                                                        b + w.cell_k, nslots);
    else
        rates_kernel<double><<<blocks, threads, 0, st>>>(M, cells, T, p, Y, ldY, dYdt, b + w.lane_r,
                                                         b + w.cell_k, nslots);
    return cudaGetLastError();
}

cudaError_t launch_rkc_table(double* tab, cudaStream_t st)
{
    rkc_table_kernel<<<(SMAX + 1 + 127) / 128, 128, 0, st>>>(tab);
    return cudaGetLastError();
}

}  // namespace kin