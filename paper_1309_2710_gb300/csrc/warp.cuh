// warp.cuh -- warp-per-cell RKC for large mechanisms (templates; instantiated
// in inst_warp_*.cu).
//
// With one lane per cell, every lane keeps its own concentrations, rates of
// progress and rate constants: ~(2 n_R + n_S) words per cell, which for
// hundreds of reactions spills out of L1/L2 and turns every f evaluation into
// a stream from HBM. Here one warp integrates one cell:
//  * the 32 lanes split the reactions (rates of progress, rounds of 32) and
//    the species (state vectors in registers: species l + 32 r in slot r of
//    lane l; stoichiometric gather over the species-major CSR);
//  * the cell's concentrations and rates of progress live in shared memory
//    (n_S + n_R words per warp); its rate constants, computed once per call
//    since T is fixed, live in the workspace cell-major and are read
//    coalesced (the working set of the resident cells stays in L2);
//  * reactions are visited in a fixed permutation (plain, then third-body,
//    then falloff) so that a round of 32 lanes mixes the dense efficiency dot
//    products with plain reactions at most once; the efficiency rows are
//    stored transposed ([species][row]) so that the lanes of a round read
//    consecutive words;
//  * all lanes follow the same cell, so the method's control flow is uniform
//    and is written as straight-line code; reductions (mixture sum, error
//    norms, spectral-radius bounds) are butterfly shuffles, which leave every
//    lane with the same bits.
// The method, its decisions and the statistics are those of the lane-per-cell
// kernel (Section 2.3 and the readings listed with it).
#pragma once
#include "kernels.cuh"
#include "seg_tables.h"

namespace kin {

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Butterfly sum over a group of G lanes (a whole warp, or a 16-lane half
// that owns one cell); mask names the group's lanes.
template <int G, typename T>
__device__ __forceinline__ T group_sum(T v, unsigned mask)
{
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
    return v;
}

template <int G>
__device__ __forceinline__ double group_max(double v, unsigned mask)
{
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(mask, v, o));
    return v;
}

__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

template <typename R>
struct EllT;
template <>
struct EllT<double> {
    __device__ static const CsrW64* tab(const MechDev& M) { return M.ell64; }
};
template <>
struct EllT<float> {
    __device__ static const CsrW32* tab(const MechDev& M) { return M.ell32; }
};

// The third-body concentration of efficiency row `row`, [M] = sum_k eff_k C_k
// (Eq. (E:rxn-rate)), summed as two interleaved partial sums (even k, odd k).
// The rows are stored 16 bytes per species group, [k / V][row][k % V] with V =
// 4 (FP32) or 2 (FP64), so that a lane reads V efficiencies with one load and
// the warp's broadcast concentrations with another; lanes of a round take
// consecutive rows, so a warp's efficiency load is one contiguous span.
template <typename R>
__device__ __forceinline__ R eff_dot(const MechDev& M, int row, const R* C);

template <>
__device__ __forceinline__ float eff_dot<float>(const MechDev& M, int row, const float* C)
{
    const int nS = M.nS, nM = M.nM, n4 = nS >> 2;
    const float4* __restrict__ a = reinterpret_cast<const float4*>(M.effV32) + row;
    const float4* c = reinterpret_cast<const float4*>(C);
    float m0 = 0.0f, m1 = 0.0f;
    for (int k = 0; k < n4; ++k) {
        const float4 e = a[(int64_t)k * nM], x = c[k];
        m0 += e.x * x.x;
        m1 += e.y * x.y;
        m0 += e.z * x.z;
        m1 += e.w * x.w;
    }
    if (nS & 3) {
        const float4 e = a[(int64_t)n4 * nM];
        const int k = n4 << 2, t = nS & 3;
        m0 += e.x * C[k];
        if (t > 1) m1 += e.y * C[k + 1];
        if (t > 2) m0 += e.z * C[k + 2];
    }
    return m0 + m1;
}

template <>
__device__ __forceinline__ double eff_dot<double>(const MechDev& M, int row, const double* C)
{
    const int nS = M.nS, nM = M.nM, n2 = nS >> 1;
    const double2* __restrict__ a = reinterpret_cast<const double2*>(M.effV64) + row;
    const double2* c = reinterpret_cast<const double2*>(C);
    double m0 = 0.0, m1 = 0.0;
    for (int k = 0; k < n2; ++k) {
        const double2 e = a[(int64_t)k * nM], x = c[k];
        m0 += e.x * x.x;
        m1 += e.y * x.y;
    }
    if (nS & 1) m0 += a[(int64_t)n2 * nM].x * C[nS - 1];
    return m0 + m1;
}

// Shared words per warp: C [nS] and Omega [nR], padded to 4, sized for FP64
// (the mixed-precision path evaluates f in FP32 for its RK stages and in FP64
// for its spectral-radius estimates, over the same words).
__host__ __device__ __forceinline__ int warp_smem_elems(const MechDev& M)
{
    return (M.nS + M.nR + 3) & ~3;
}

// The cell's rate constants in shared memory too: f reads every k_j once per
// evaluation, and staged behind C and Omega that read is a shared load instead
// of an L2 round trip on the f's critical path. Isothermal only (with the
// energy equation k follows T inside f), and only for small mechanisms, whose
// group words stay within WARP_K_SMEM_MAX_BYTES: shared memory comes out of
// the same on-chip array as L1, and for 53 species / 634 reactions the larger
// carve-out cost more in L1 misses (tables, spills) than the staged k saved
// (163 K vs 174 K cells/s on GB300), while 9 species / 38 reactions gained.
constexpr int WARP_K_SMEM_MAX_BYTES = 2048;

template <typename R, bool EN>
__host__ __device__ __forceinline__ int warp_k_words(const MechDev& M)
{
    if (EN) return 0;
    const int kw = ((M.nR + M.nFO) * (int)sizeof(R) + 7) / 8;
    return (warp_smem_elems(M) + kw) * 8 <= WARP_K_SMEM_MAX_BYTES ? kw : 0;
}

// Shared FP64 words per cell group: C and Omega, then the staged k (if any).
template <typename R, bool EN>
__host__ __device__ __forceinline__ int warp_group_words(const MechDev& M)
{
    return warp_smem_elems(M) + warp_k_words<R, EN>(M);
}

// f for the warp's cell (Eqs. (E:mass), (E:spec-rate), (E:rxn-rate)) in
// arithmetic type R. Kc are the cell's rate constants (stored as KT) in
// reaction-permutation order followed by k0/kinf per falloff ordinal (written
// earlier in the same pre-pass kernel, so not read through the read-only
// cache); C and OM are the warp's shared arrays. Ctot and invCtot (the total
// concentration p / (R T) and its reciprocal) come in the arithmetic type, so
// that the FP32 evaluation's scalar work stays off the FP64 pipe: only the
// state's conversions in and the rates' conversions out are FP64 operations.
template <typename R, typename KT, int NR, int G = 32>
__device__ __forceinline__ void warp_feval(const MechDev& M, const KT* Kc, R* C, R* OM,
                                           R Ctot, R invCtot, const double (&x)[NR],
                                           double (&out)[NR], int lane, unsigned mask = 0xffffffffu)
{
    const int nS = M.nS, nR = M.nR, nM = M.nM;
    const R* __restrict__ invW = Tab<R>::invW(M);
    R s = R(0);
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const int i = lane + G * r;
        if (i < nS) {
            const R m = (R)x[r] * invW[i];
            C[i] = m;
            s += m;
        }
    }
    s = group_sum<G>(s, mask);
    const R rho = Ctot * Tab<R>::inv(s);
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const int i = lane + G * r;
        if (i < nS) C[i] = C[i] * rho;
    }
    __syncwarp(mask);
    // permutation order: plain reactions, then third-body (efficiency row
    // q - nP), then falloff (ordinal q - nF)
    const int nP = nR - nM, nF = nR - M.nFO;
    const uint32_t* __restrict__ rxw = M.rxw;
#pragma unroll 1
    for (int q = lane; q < nR; q += G) {
        const uint32_t w = rxw[q];
        R v = (R)Kc[q];
        const int r0 = (int)(w & 0xffffu) - 1, r1 = (int)(w >> 16) - 1;
        if (r0 >= 0) v *= C[r0];
        if (r1 >= 0) v *= C[r1];
        if (q >= nP) {
            const R Mc = eff_dot<R>(M, q - nP, C);
            if (q < nF) {
                v *= Mc;
            } else {
                const R Pr = (R)Kc[nR + (q - nF)] * Mc;
                v *= rdiv<R>(Pr, R(1) + Pr);
            }
        }
        OM[q] = v;
    }
    __syncwarp(mask);
    const R invrho = s * invCtot;
    if constexpr (G == 32 && sizeof(R) == 4) {
        if (M.seg_ent) {
            // omega over equal chunks of the nonzeros (seg_tables.h); the
            // partial sums land past Omega, in the FP32 half of the warp's
            // words that only the FP64 evaluations use
            float* P = reinterpret_cast<float*>(OM) + nR;
            const uint32_t* __restrict__ ent = M.seg_ent + lane;
            int slot = M.seg_slot0[lane];
            float w = 0.0f;
            const int K = M.seg_K;
            for (int k = 0; k < K; ++k) {
                const uint32_t e = ent[32 * k];
                w = fmaf(__uint_as_float(e & SEG_NU_MASK), OM[e & SEG_POS_MASK], w);
                if (e & SEG_FLUSH) {
                    P[slot++] = w;
                    w = 0.0f;
                }
            }
            __syncwarp(mask);
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const int i = lane + 32 * r;
                double o = 0.0;
                if (i < nS) {
                    const int pt = M.seg_part[i];
                    if (pt >= 0) {
                        const float* pp = P + (pt >> 8);
                        float v = pp[0];
                        for (int c = 1; c < (pt & 0xff); ++c) v += pp[c];
                        o = (double)(v * (M.W32[i] * invrho));
                    }
                }
                out[r] = o;
            }
            __syncwarp(mask);  // C, OM and P are rewritten by the next evaluation
            return;
        }
    }
    // W_i omega_i over the species' row (W_i folded into its coefficients).
    // With 32 lanes per cell the row is read from the ELL copy, where the
    // lanes of a step read consecutive entries (one or two cache lines per
    // load instead of one line per lane); the entries and their order are
    // those of the species-major rows.
    const R* __restrict__ nuW = Tab<R>::nuW(M);
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const int i = lane + G * r;
        double o = 0.0;
        if (i < nS) {
            R w0 = R(0), w1 = R(0);
            if constexpr (G == 32) {
                const int len = M.csr_ptr[i + 1] - M.csr_ptr[i];
                const auto* __restrict__ p = EllT<R>::tab(M) + M.ell_base[r] + lane;
                int k = 0;
                for (; k + 1 < len; k += 2) {
                    const auto a = p[32 * k], b = p[32 * (k + 1)];
                    w0 += a.nuW * OM[a.pos];
                    w1 += b.nuW * OM[b.pos];
                }
                if (k < len) {
                    const auto a = p[32 * k];
                    w0 += a.nuW * OM[a.pos];
                }
            } else {
                const int e1 = M.csr_ptr[i + 1];
                int e = M.csr_ptr[i];
                for (; e + 1 < e1; e += 2) {
                    w0 += nuW[e] * OM[M.csrp_rxn[e]];
                    w1 += nuW[e + 1] * OM[M.csrp_rxn[e + 1]];
                }
                if (e < e1) w0 += nuW[e] * OM[M.csrp_rxn[e]];
            }
            o = (double)((w0 + w1) * invrho);
        }
        out[r] = o;
    }
    __syncwarp(mask);  // C and OM are rewritten by the next evaluation
}

// Element r of a register vector for a warp-uniform r.
template <int NR>
__device__ __forceinline__ double reg_get(const double (&v)[NR], int r);

// f with the energy equation (Eqs. (E:mass), (E:energy)) for the warp's cell:
// state component nS is T (lane nS % 32, slot nS / 32). Each lane computes the
// rate constants of its reactions from T (they follow T at every
// evaluation); the enthalpy sum and the mixture heat capacity are FP64 warp
// sums, and dT/dt lands in T's slot.
template <typename R, int NR, int G = 32>
__device__ __forceinline__ void warp_feval_energy(const MechDev& M, double p, R* C, R* OM,
                                                  const double (&x)[NR], double (&out)[NR], int lane,
                                                  unsigned mask = 0xffffffffu)
{
    const int nS = M.nS, nR = M.nR, nM = M.nM;
    const double T = __shfl_sync(mask, reg_get(x, nS / G), nS % G, G);
    const double lnT = log(T), invT = ddiv(1.0, T);
    const double Ctot = p * 1e-6 * invT * (1.0 / R_GAS), invCtot = ddiv(1.0, Ctot);
    const R* __restrict__ invW = Tab<R>::invW(M);
    R s = R(0);
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const int i = lane + G * r;
        if (i < nS) {
            const R m = (R)x[r] * invW[i];
            C[i] = m;
            s += m;
        }
    }
    s = group_sum<G>(s, mask);
    const R rho = (R)Ctot * Tab<R>::inv(s);
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const int i = lane + G * r;
        if (i < nS) C[i] = C[i] * rho;
    }
    __syncwarp(mask);
    const int nP = nR - nM, nF = nR - M.nFO;
    const uint32_t* __restrict__ rxw = M.rxw;
    for (int q = lane; q < nR; q += G) {
        const uint32_t w = rxw[q];
        const int j = M.rxn_perm[q];
        const double a = M.lnA[j] + M.beta[j] * lnT - M.EaR[j] * invT;
        R v = Tab<R>::ex(a);
        const int r0 = (int)(w & 0xffffu) - 1, r1 = (int)(w >> 16) - 1;
        if (r0 >= 0) v *= C[r0];
        if (r1 >= 0) v *= C[r1];
        if (q >= nP) {
            const R Mc = eff_dot<R>(M, q - nP, C);
            if (q < nF) {
                v *= Mc;
            } else {
                const double a0 = M.lnA0[j] + M.beta0[j] * lnT - M.Ea0R[j] * invT;
                const R Pr = Tab<R>::ex(a0 - a) * Mc;
                v *= rdiv<R>(Pr, R(1) + Pr);
            }
        }
        OM[q] = v;
    }
    __syncwarp(mask);
    const R* __restrict__ nu = Tab<R>::nu(M);
    const double invrho = (double)s * invCtot, dT = T - T_REF;
    double hw = 0.0, cpm = 0.0;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const int i = lane + G * r;
        double o = 0.0;
        if (i < nS) {
            R w0 = R(0), w1 = R(0);
            const int e1 = M.csr_ptr[i + 1];
            int e = M.csr_ptr[i];
            for (; e + 1 < e1; e += 2) {
                w0 += nu[e] * OM[M.csrp_rxn[e]];
                w1 += nu[e + 1] * OM[M.csrp_rxn[e + 1]];
            }
            if (e < e1) w0 += nu[e] * OM[M.csrp_rxn[e]];
            const double om = (double)(w0 + w1);
            o = om * (M.W[i] * invrho);
            hw += (M.Hf[i] + M.cp[i] * dT) * om;
            cpm += x[r] * M.cpW[i];
        }
        out[r] = o;
    }
    hw = group_sum<G>(hw, mask);
    cpm = group_sum<G>(cpm, mask);
    const double dTdt = ddiv(-hw * invrho, cpm);
#pragma unroll
    for (int r = 0; r < NR; ++r)
        if (lane + G * r == nS) out[r] = dTdt;
    __syncwarp(mask);  // C and OM are rewritten by the next evaluation
}

// Element r of a register vector for a warp-uniform r.
template <int NR>
__device__ __forceinline__ double reg_get(const double (&v)[NR], int r)
{
    double o = v[0];
#pragma unroll
    for (int q = 1; q < NR; ++q)
        if (r == q) o = v[q];
    return o;
}

template <typename R, int NR, bool EN>
struct WarpRKC {
    const Launch& L;
    const MechDev& M;
    R* C;
    R* OM;
    double* C64;   // the same shared words as C and OM, for the FP64 evaluations
    double* OM64;
    R* Ks;         // the warp's staged rate constants, or null
    const R* Kc;
    int lane, nV;  // nV: state length, nS + 1 with the energy equation
    double Ctot, invCtot, atol, rtol, p;
    R CtotR, invCtotR;   // the same in the rate type
    int nfe, nsig, nfs;  // f evaluations, sigma estimates, f evaluations inside them
    double y[NR], f0[NR], w1[NR], w2[NR], fx[NR], x[NR], ev[NR];

    __device__ explicit WarpRKC(const Launch& l) : L(l), M(l.M), Kc(nullptr), lane(threadIdx.x & 31), nV(l.nV)
    {
        C64 = reinterpret_cast<double*>(kin_smem) + (size_t)(threadIdx.x >> 5) * warp_group_words<R, EN>(M);
        OM64 = C64 + M.nS;
        C = reinterpret_cast<R*>(C64);
        OM = C + M.nS;
        Ks = warp_k_words<R, EN>(M) ? reinterpret_cast<R*>(C64 + warp_smem_elems(M)) : nullptr;
    }

    __device__ __forceinline__ bool valid(int r) const { return lane + 32 * r < nV; }

    __device__ __forceinline__ void f(const double (&in)[NR], double (&o)[NR])
    {
        if constexpr (EN) warp_feval_energy<R, NR>(M, p, C, OM, in, o, lane);
        else warp_feval<R, R, NR>(M, Kc, C, OM, CtotR, invCtotR, in, o, lane);
        nfe++;
    }

    // f in FP64 for the spectral-radius estimates (FP32 rounding noise in
    // f(y + v) - f(y) would swamp the difference; see SIG_SQRT_U).
    __device__ __forceinline__ void fs(const double (&in)[NR], double (&o)[NR])
    {
        if constexpr (EN)
            warp_feval_energy<double, NR>(M, p, C64, OM64, in, o, lane);
        else if constexpr (sizeof(R) == 4)
            warp_feval<double, R, NR>(M, Kc, C64, OM64, Ctot, invCtot, in, o, lane);
        else
            warp_feval<double, double, NR>(M, Kc, C, OM, Ctot, invCtot, in, o, lane);
        nfe++;
        nfs++;
    }

    // Weighted RMS norm, Eq. (E:rmsE), of d with T_i = atol + rtol max(|a_i|, |b_i|).
    __device__ double rms(const double (&d)[NR], const double (&a)[NR], const double (&b)[NR]) const
    {
        double acc = 0.0;
#pragma unroll
        for (int r = 0; r < NR; ++r)
            if (valid(r)) {
                const double sc = atol + rtol * fmax(fabs(a[r]), fabs(b[r]));
                const double q = ddiv(d[r], sc);
                acc += q * q;
            }
        return dsqrt(ddiv(warp_sum(acc), (double)nV));
    }

    // FP64 f(y), the base of the spectral-radius differences: f0 in the FP64
    // path; in the mixed-precision path w2, which the estimate evaluates first.
    __device__ __forceinline__ double sig_base(int r) const
    {
        if constexpr (sizeof(R) == 4) return w2[r];
        else return f0[r];
    }

    // Start of the nonlinear power method, warm-started from ev: scales ev to
    // the difference length sqrt(u) |y| and returns that length.
    __device__ double power_setup()
    {
        double yn = 0.0, vn = 0.0;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            yn += y[r] * y[r];
            vn += ev[r] * ev[r];
        }
        yn = dsqrt(warp_sum(yn));
        vn = dsqrt(warp_sum(vn));
        const double dyn = yn > 0.0 ? SIG_SQRT_U * yn : SIG_SQRT_U;
        if (!(vn > 0.0) || !isfinite(vn)) {
#pragma unroll
            for (int r = 0; r < NR; ++r) ev[r] = valid(r) ? 1.0 : 0.0;
            vn = dsqrt((double)nV);
        }
        const double sc0 = ddiv(dyn, vn);
#pragma unroll
        for (int r = 0; r < NR; ++r) ev[r] = ev[r] * sc0;
        return dyn;
    }

    // Spectral radius at y: the Gershgorin bound on the finite-difference
    // Jacobian (one column per evaluation) or the nonlinear power method
    // warm-started from ev (at most 20 products, stopping when two estimates
    // agree to 1 %; returns 1.2 times the last), Section 2.3. The mixed-
    // precision path first re-evaluates f(y) in FP64 into w2. `first` starts
    // the power method from f(y). Every FP64 evaluation of the estimate goes
    // through the one call of fs below, so the kernel holds one inlined copy
    // of the FP64 f.
    __device__ double sigma(bool first)
    {
        constexpr bool MIX = sizeof(R) == 4;
        const bool pw = L.sigma_method == KIN_SIGMA_POWER;
        double rs[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) rs[r] = 0.0;
        double dyn = 0.0, sig = 0.0, prev = 0.0, eps = 0.0;
        if constexpr (!MIX) {
            if (first)
#pragma unroll
                for (int r = 0; r < NR; ++r) ev[r] = f0[r];
            if (pw) dyn = power_setup();
        }
        for (int k = MIX ? -1 : 0;; ++k) {  // k = -1: the base f(y)
            if (k < 0) {
#pragma unroll
                for (int r = 0; r < NR; ++r) x[r] = y[r];
            } else if (pw) {
#pragma unroll
                for (int r = 0; r < NR; ++r) x[r] = y[r] + ev[r];
            } else {  // Gershgorin column k
                const int kr = k >> 5, kl = k & 31;
                const double yk = __shfl_sync(0xffffffffu, reg_get(y, kr), kl);
                eps = SIG_SQRT_U * fmax(fabs(yk), atol);
#pragma unroll
                for (int r = 0; r < NR; ++r) x[r] = (r == kr && lane == kl) ? yk + eps : y[r];
            }
            fs(x, fx);
            if (k < 0) {
#pragma unroll
                for (int r = 0; r < NR; ++r) w2[r] = fx[r];
                if (first)
#pragma unroll
                    for (int r = 0; r < NR; ++r) ev[r] = w2[r];
                if (pw) dyn = power_setup();
                continue;
            }
            if (pw) {
                double wn = 0.0;
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    fx[r] = fx[r] - sig_base(r);
                    wn += fx[r] * fx[r];
                }
                wn = dsqrt(warp_sum(wn));
                sig = ddiv(wn, dyn);
                if (!(wn > 0.0) || !isfinite(wn)) break;
                const double sc = ddiv(dyn, wn);
#pragma unroll
                for (int r = 0; r < NR; ++r) ev[r] = fx[r] * sc;
                if (k >= 1 && fabs(sig - prev) <= 0.01 * sig) break;
                prev = sig;
                if (k + 1 >= 20) break;
            } else {
                const double ie = rcp_newton(eps);
#pragma unroll
                for (int r = 0; r < NR; ++r)
                    if (valid(r)) rs[r] += fabs((fx[r] - sig_base(r)) * ie);
                if (k + 1 >= nV) {
                    double m = 0.0;
#pragma unroll
                    for (int r = 0; r < NR; ++r) m = fmax(m, rs[r]);
                    return warp_max(m);
                }
            }
        }
        return 1.2 * sig;
    }

    __device__ __forceinline__ const double* coef(int s, int j) const
    {
        return M.rkc + ((int64_t)s * RKC_TAB_S + j) * RKC_TAB_W;
    }

    // RKC integration over [0, dt] from the pre-pass state (y, f0, ev and the
    // given sigma and first trial step h). Returns the cell status.
    __device__ int run(double dt, double sig, double h, int& nacc, int& nrej)
    {
        double t = 0.0, hprev = 0.0, cprev = 0.0;
        int attempts = 0, since = 0;
        bool sigma_here = true, last_rej = false, have_prev = false;
        const double invN = ddiv(1.0, (double)nV);
        for (;;) {
            if (attempts >= L.max_steps) return KIN_CELL_MAXSTEPS;
            if (since >= 25 || (last_rej && !sigma_here)) {
                sig = sigma(false);
                nsig++;
                since = 0;
                sigma_here = true;
                if (!isfinite(sig)) return KIN_CELL_NONFINITE;
            }
            double hh = h;
            bool last = false;
            if (hh >= dt - t) {
                hh = dt - t;
                last = true;
            }
            // The mixed-precision path takes the stage count's square root in
            // FP32: s is an integer, which the FP32 root changes only where
            // 1 + sqrt(1 + 1.54 h sigma) lies within FP32 rounding of an
            // integer, and the FP64 root is a dozen instructions on the FP64
            // pipe that all 32 lanes repeat.
            double sr;
            if constexpr (sizeof(R) == 4)
                sr = (double)floorf(1.0f + sqrtf(1.0f + (float)(1.54 * hh * sig)));
            else
                sr = floor(1.0 + dsqrt(1.0 + 1.54 * hh * sig));
            int s;
            if (sr < 2.0) {
                s = 2;
            } else if (sr > (double)SMAX) {
                s = SMAX;
                hh = ddiv((SMAX - 1.0) * (SMAX - 1.0) - 1.0, 1.54 * sig);
                last = false;
            } else {
                s = (int)sr;
            }
            // w_0 = y, w_1 = y + mu~_1 h f_0, then the three-term recursion
            const double m1 = coef(s, 1)[2] * hh;
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                w2[r] = y[r];
                w1[r] = y[r] + m1 * f0[r];
            }
            for (int j = 2;; ++j) {
                f(w1, fx);  // f(w_{j-1}); after the last stage, f(w_s)
                if (j > s) break;
                const double* c = coef(s, j);
                const double mu = c[0], nu = c[1], mt = c[2] * hh, gt = c[3] * hh, c0 = c[4];
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    const double wn = c0 * y[r] + mu * w1[r] + nu * w2[r] + mt * fx[r] + gt * f0[r];
                    w2[r] = w1[r];
                    w1[r] = wn;
                }
            }
            attempts++;
            double acc = 0.0;
#pragma unroll
            for (int r = 0; r < NR; ++r)
                if (valid(r)) {
                    const double d = 0.8 * (y[r] - w1[r]) + 0.4 * hh * (f0[r] + fx[r]);
                    const double sc = atol + rtol * fmax(fabs(y[r]), fabs(w1[r]));
                    const double q = d * rcp_newton(sc);
                    acc += q * q;
                }
            // x = ||Delta||^2; z = x^(-1/6) = err^(-1/3) (see the lane kernel)
            // (one evaluation of the power serves both branches)
            const double xe = warp_sum(acc) * invN;
            // (the mixed-precision path keeps the FP32 power, within 4 ulp: a
            // step-size factor, with the FP32 rates' precision)
            double z = 0.0;
            if (xe > 0.0 && isfinite(xe)) {
                if constexpr (sizeof(R) == 4)
                    z = f32_normal(xe) ? (double)powf((float)xe, -1.0f / 6.0f) : dpow(xe, -1.0 / 6.0);
                else
                    z = rpow6_newton(xe);
            }
            if (xe <= 1.0) {
                nacc++;
                double fac, c3 = 0.0;
                if (xe == 0.0) {
                    fac = 10.0;
                } else {
                    const double z2 = z * z;
                    c3 = xe * (z2 * z2 * z);
                    if (have_prev && !last_rej && cprev > 0.0)
                        fac = 0.8 * hh * cprev * z2 * rcp_newton(hprev);
                    else fac = 0.8 * z;
                }
                fac = fmin(10.0, fmax(0.1, fac));
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    y[r] = w1[r];
                    f0[r] = fx[r];
                }
                if (last) return KIN_CELL_OK;
                t += hh;
                have_prev = true;
                hprev = hh;
                cprev = c3;
                last_rej = false;
                sigma_here = false;
                since++;
                h = fac * hh;
            } else {
                nrej++;
                double fac = isfinite(xe) ? 0.8 * z : 0.1;
                if (fac < 0.1) fac = 0.1;
                last_rej = true;
                h = fac * hh;
                if (h < 1e-20 * dt) return KIN_CELL_HMIN;
            }
        }
    }
};

// Register budget at 256 threads per block. OCC 0: 128 registers (no spills
// for up to 4 vector slots; 16 resident warps per SM); OCC 1, for 2 or fewer
// slots: 48 registers (40 warps per SM, about the most that the shared words
// of a 53-species / 634-reaction cell leave room for; some values spill to
// local memory), or 80 (24 warps) with the energy equation, whose f holds
// more live values; 128 for 4 and 8 slots. The isothermal f evaluation of
// these mechanisms waits on L1 and shared-memory round trips, and more
// resident warps hide more of that latency: on 53 species / 634 reactions,
// mixed precision, 198 K cells/s at 32 warps per SM (64 registers), 217 K at
// 36 (56) and 237 K at 40 (48), against 178 K at 24 (80). With the energy
// equation 74.1 K at 80 registers against 72.1 K at 64.
template <int NR, int OCC, bool EN>
struct WarpBounds {
    static constexpr int min_blocks = NR == 8 ? (OCC ? 2 : 1) : (OCC && NR <= 2 ? (EN ? 3 : 5) : 2);
};

// Pre-pass, one warp per cell (grid-stride over cells): the cell's rate
// constants (stored cell-major for the main kernel), f(y0), sigma and the
// initial step h1 (Section 2.3).
template <typename R, int NR, int OCC, bool EN>
__global__ void __launch_bounds__(256, WarpBounds<NR, OCC, EN>::min_blocks) warp_init_kernel(const __grid_constant__ Launch L)
{
    WarpRKC<R, NR, EN> W(L);
    const MechDev& M = L.M;
    const int lane = W.lane, nK = M.nR + M.nFO, nS = M.nS, nV = L.nV;
    const int64_t nwarps = L.nslots >> 5;
    for (int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < L.total; g += nwarps) {
        const int ii = find_inst(L, g);
        const InstDev& I = L.inst[ii];
        const int64_t c = g - L.start[ii];
        const double T = I.T[c], p = I.p[c];
        W.Ctot = ddiv(p * 1e-6, R_GAS * T);
        W.invCtot = ddiv(1.0, W.Ctot);
        W.CtotR = (R)W.Ctot;
        W.invCtotR = (R)W.invCtot;
        W.atol = I.atol;
        W.rtol = I.rtol;
        W.p = p;
        W.nfe = 0;
        W.nfs = 0;
        if constexpr (!EN) {
            // rate constants (Eq. (E:rxn-const)) in permutation order; with the
            // energy equation they follow T and are formed inside f instead
            // (for the main kernel in the workspace, and for this kernel's own
            // evaluations in the staged copy when there is one)
            R* kc = reinterpret_cast<R*>(L.cell_k) + g * nK;
            R* ks = W.Ks ? W.Ks : kc;
            const double lnT = log(T), invT = ddiv(1.0, T);
            for (int q = lane; q < M.nR; q += 32) {
                const int j = M.rxn_perm[q];
                const double a = M.lnA[j] + M.beta[j] * lnT - M.EaR[j] * invT;
                const R k = Tab<R>::ex(a);
                kc[q] = k;
                ks[q] = k;
                const int fo = M.rxnp[q].fo;
                if (fo >= 0) {
                    const double a0 = M.lnA0[j] + M.beta0[j] * lnT - M.Ea0R[j] * invT;
                    const R k0 = Tab<R>::ex(a0 - a);
                    kc[M.nR + fo] = k0;
                    ks[M.nR + fo] = k0;
                }
            }
            __syncwarp();
            W.Kc = ks;
        }
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const int i = lane + 32 * r;
            W.y[r] = i < nS ? I.Y[(int64_t)i * I.ldY + c] : (i == nS && EN ? T : 0.0);
        }
        W.f(W.y, W.f0);
        bool fin = true;
#pragma unroll
        for (int r = 0; r < NR; ++r) fin &= isfinite(W.f0[r]);
        fin = __all_sync(0xffffffffu, fin);
        uint8_t st = fin ? 0 : KIN_CELL_NONFINITE;
        double sig = 0.0, h = I.dt;
        if (fin) {
            sig = W.sigma(true);
            if (!isfinite(sig)) {
                st = KIN_CELL_NONFINITE;
            } else {
                double h0 = sig > 0.0 ? ddiv(1.0, sig) : I.dt;
                if (h0 > I.dt) h0 = I.dt;
#pragma unroll
                for (int r = 0; r < NR; ++r) W.x[r] = W.y[r] + h0 * W.f0[r];
                W.f(W.x, W.fx);
#pragma unroll
                for (int r = 0; r < NR; ++r) W.x[r] = h0 * (W.fx[r] - W.f0[r]);  // Delta_0
                const double e0 = W.rms(W.x, W.y, W.y);
                if (!isfinite(e0)) h = 0.1 * h0;
                else h = e0 > 0.0 ? ddiv(0.1 * h0, dsqrt(e0)) : I.dt;
                if (h > I.dt) h = I.dt;
                if (h < 1e-20 * I.dt) st = KIN_CELL_HMIN;
            }
        }
#pragma unroll
        for (int r = 0; r < NR; ++r)
            if (W.valid(r)) {
                L.cell_f0[g * nV + lane + 32 * r] = W.f0[r];
                if (L.cell_ev) L.cell_ev[g * nV + lane + 32 * r] = W.ev[r];
            }
        if (lane == 0) {
            L.cell_sig[g] = sig;
            L.cell_h[g] = h;
            L.cell_nfe[g] = W.nfe;
            L.cell_nfs[g] = W.nfs;
            L.cell_st[g] = st;
        }
    }
}

// Persistent main kernel: each warp takes cells from the queue in the
// longest-first order and integrates them one after another.
template <typename R, int NR, int OCC, bool EN>
__global__ void __launch_bounds__(256, WarpBounds<NR, OCC, EN>::min_blocks) warp_integrate_kernel(const __grid_constant__ Launch L)
{
    WarpRKC<R, NR, EN> W(L);
    const MechDev& M = L.M;
    const int lane = W.lane, nK = M.nR + M.nFO, nS = M.nS, nV = L.nV;
    for (;;) {
        unsigned long long q = 0;
        if (lane == 0) q = atomicAdd(L.queue, 1ull);
        q = __shfl_sync(0xffffffffu, q, 0);
        if (q >= (unsigned long long)L.total) return;
        const int64_t g = L.order[q];
        const int ii = find_inst(L, g);
        const InstDev& I = L.inst[ii];
        const int64_t c = g - L.start[ii];
        int nacc = 0, nrej = 0, code;
        W.nfe = L.cell_nfe[g];
        W.nfs = L.cell_nfs[g];
        W.nsig = 1;
        const uint8_t pre = L.cell_st[g];
        if (pre != 0) {
            code = pre;  // decided by the pre-pass; Y stays as given
        } else {
            const double T = I.T[c], p = I.p[c];
            W.Ctot = ddiv(p * 1e-6, R_GAS * T);
            W.invCtot = ddiv(1.0, W.Ctot);
            W.CtotR = (R)W.Ctot;
            W.invCtotR = (R)W.invCtot;
            W.atol = I.atol;
            W.rtol = I.rtol;
            W.p = p;
            if constexpr (EN) {
                W.Kc = nullptr;
            } else {
                const R* kg = reinterpret_cast<const R*>(L.cell_k) + g * nK;
                if (W.Ks) {  // stage the cell's k (the last f of the previous cell ended in a sync)
                    for (int q = lane; q < nK; q += 32) W.Ks[q] = kg[q];
                    __syncwarp();
                    W.Kc = W.Ks;
                } else {
                    W.Kc = kg;
                }
            }
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const int i = lane + 32 * r;
                const bool v = i < nV;
                W.y[r] = i < nS ? I.Y[(int64_t)i * I.ldY + c] : (v ? T : 0.0);
                W.f0[r] = v ? L.cell_f0[g * nV + i] : 0.0;
                W.ev[r] = (v && L.cell_ev) ? L.cell_ev[g * nV + i] : 0.0;
            }
            code = W.run(I.dt, L.cell_sig[g], L.cell_h[g], nacc, nrej);
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const int i = lane + 32 * r;
                if (i < nS) I.Y[(int64_t)i * I.ldY + c] = W.y[r];
                else if (i == nS && EN) I.T[c] = W.y[r];
            }
        }
        if (lane == 0) {
            if (I.status) I.status[c] = (uint8_t)code;
            if (I.stats) {
                int32_t* st = I.stats + KIN_NSTATS * c;
                st[0] = W.nfe;
                st[1] = nacc;
                st[2] = nrej;
                st[3] = W.nsig;
                st[4] = W.nfs;
            }
        }
    }
}

template <typename R, bool EN>
inline size_t warp_smem_bytes(const MechDev& M, int threads)
{
    return (size_t)warp_group_words<R, EN>(M) * (threads / 32) * 8;
}

// ---------------------------------------------------- RKCK, warp per cell --
// Cash-Karp 5(4) with the step rule of Section 2.2 (Table 1, Eq. (E:hnew)),
// one group of G lanes per cell (G = 32, a warp; or G = 16, two cells per
// warp, for states of at most 16 components, where a whole warp would leave
// most of its FP64 lanes idle), in one persistent kernel: RKCK needs no
// spectral radius or initial-step estimate, so there is no pre-pass and no
// cost ordering. A group takes the next cell, forms its rate constants
// (cell-major in the workspace, unless they follow T with the energy
// equation) and integrates it with straight-line control flow; the decisions
// are those of the lane-per-cell kernel. Every collective of a group names
// only the group's lanes, so the two halves of a warp may diverge.
template <typename R, int NR, bool EN, int G>
struct WarpRKCK {
    const Launch& L;
    const MechDev& M;
    R* C;
    R* OM;
    R* Ks;  // the group's staged rate constants, or null
    const R* Kc;
    int lane, nV;
    unsigned mask;  // the group's lanes
    double Ctot, invCtot, atol, rtol, p;
    R CtotR, invCtotR;  // the same in the rate type
    int nfe;
    double y[NR], x[NR], kx[NR], k[6][NR];

    __device__ explicit WarpRKCK(const Launch& l)
        : L(l), M(l.M), Kc(nullptr), lane(threadIdx.x & (G - 1)), nV(l.nV),
          mask(G == 32 ? 0xffffffffu : (0xffffu << (threadIdx.x & 16)))
    {
        double* base = reinterpret_cast<double*>(kin_smem) + (size_t)(threadIdx.x / G) * warp_group_words<R, EN>(M);
        C = reinterpret_cast<R*>(base);
        OM = C + M.nS;
        Ks = warp_k_words<R, EN>(M) ? reinterpret_cast<R*>(base + warp_smem_elems(M)) : nullptr;
    }

    __device__ __forceinline__ bool valid(int r) const { return lane + G * r < nV; }

    __device__ __forceinline__ void f(const double (&in)[NR], double (&o)[NR])
    {
        if constexpr (EN) warp_feval_energy<R, NR, G>(M, p, C, OM, in, o, lane, mask);
        else warp_feval<R, R, NR, G>(M, Kc, C, OM, CtotR, invCtotR, in, o, lane, mask);
        nfe++;
    }

    // Integrate over [0, dt] from y with k[0] = f(y); returns the cell status.
    __device__ int run(double dt, int& nacc, int& nrej)
    {
        double t = 0.0, h = dt;  // first trial step: the whole flow step
        int attempts = 0;
        for (;;) {
            if (attempts >= L.max_steps) return KIN_CELL_MAXSTEPS;
            double hh = h;
            bool last = false;
            if (hh >= dt - t) {
                hh = dt - t;
                last = true;
            }
            for (int st = 1; st < 6; ++st) {  // stage points y + hh sum_l b_{st,l} k_l
                // (stage indices are resolved with unrolled selects, so k stays
                // in registers)
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    double acc = 0.0;
#pragma unroll
                    for (int l = 0; l < 5; ++l)
                        if (l < st) acc += CK_B[st][l] * k[l][r];
                    x[r] = y[r] + hh * acc;
                }
                f(x, kx);
#pragma unroll
                for (int l = 1; l < 6; ++l)
                    if (l == st)
#pragma unroll
                        for (int r = 0; r < NR; ++r) k[l][r] = kx[r];
            }
            double errmax = 0.0;
            bool blown = false;
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                double s5 = 0.0, e = 0.0;
#pragma unroll
                for (int l = 0; l < 6; ++l) {
                    s5 += CK_C[l] * k[l][r];
                    e += CK_E[l] * k[l][r];
                }
                x[r] = y[r] + hh * s5;
                if (valid(r)) {
                    const double tol = rtol * (fabs(y[r]) + fabs(hh * k[0][r])) + atol;
                    const double q = fabs(hh * e) * rcp_newton(tol);
                    blown |= isnan(q);
                    if (q > errmax) errmax = q;
                }
            }
            // group maximum; a NaN component makes the estimate non-finite
            errmax = group_max<G>(errmax, mask);
            if (__any_sync(mask, blown)) errmax = __longlong_as_double(0x7ff8000000000000ll);
            attempts++;
            if (errmax <= 1.0) {
                nacc++;
#pragma unroll
                for (int r = 0; r < NR; ++r) y[r] = x[r];
                if (last) return KIN_CELL_OK;
                t += hh;
                const double hn = errmax == 0.0 ? 5.0 * hh : 0.9 * hh * rpow5_newton(errmax);
                h = fmin(hn, 5.0 * hh);
                f(y, k[0]);
                bool fin = true;
#pragma unroll
                for (int r = 0; r < NR; ++r) fin &= isfinite(k[0][r]);
                if (!__all_sync(mask, fin)) return KIN_CELL_NONFINITE;
            } else {
                nrej++;
                const double hn = isfinite(errmax) ? 0.9 * hh * rpow4_newton(errmax) : 0.1 * hh;
                h = fmax(hn, 0.1 * hh);
                if (h < 1e-20 * dt) return KIN_CELL_HMIN;
            }
        }
    }
};

template <typename R, int NR, bool EN, int G>
__global__ void __launch_bounds__(256, NR == 8 ? 1 : 2) warp_rkck_kernel(const __grid_constant__ Launch L)
{
    WarpRKCK<R, NR, EN, G> W(L);
    const MechDev& M = L.M;
    const int lane = W.lane, nK = M.nR + M.nFO, nS = M.nS;
    for (;;) {
        unsigned long long q = 0;
        if (lane == 0) q = atomicAdd(L.queue, 1ull);
        q = __shfl_sync(W.mask, q, 0, G);
        if (q >= (unsigned long long)L.total) return;
        const int64_t g = (int64_t)q;
        const int ii = find_inst(L, g);
        const InstDev& I = L.inst[ii];
        const int64_t c = g - L.start[ii];
        const double T = I.T[c], p = I.p[c];
        W.Ctot = ddiv(p * 1e-6, R_GAS * T);
        W.invCtot = ddiv(1.0, W.Ctot);
        W.CtotR = (R)W.Ctot;
        W.invCtotR = (R)W.invCtot;
        W.atol = I.atol;
        W.rtol = I.rtol;
        W.p = p;
        W.nfe = 0;
        if constexpr (!EN) {
            // formed straight into the staged copy when there is one (the
            // previous cell's last f ended in a sync of the group)
            R* kc = W.Ks ? W.Ks : reinterpret_cast<R*>(L.cell_k) + g * nK;
            const double lnT = log(T), invT = ddiv(1.0, T);
            for (int qq = lane; qq < M.nR; qq += G) {
                const int j = M.rxn_perm[qq];
                const double a = M.lnA[j] + M.beta[j] * lnT - M.EaR[j] * invT;
                kc[qq] = Tab<R>::ex(a);
                const int fo = M.rxnp[qq].fo;
                if (fo >= 0) {
                    const double a0 = M.lnA0[j] + M.beta0[j] * lnT - M.Ea0R[j] * invT;
                    kc[M.nR + fo] = Tab<R>::ex(a0 - a);
                }
            }
            __syncwarp(W.mask);
            W.Kc = kc;
        }
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const int i = lane + G * r;
            W.y[r] = i < nS ? I.Y[(int64_t)i * I.ldY + c] : (i == nS && EN ? T : 0.0);
        }
        W.f(W.y, W.k[0]);
        bool fin = true;
#pragma unroll
        for (int r = 0; r < NR; ++r) fin &= isfinite(W.k[0][r]);
        int nacc = 0, nrej = 0, code = KIN_CELL_NONFINITE;
        if (__all_sync(W.mask, fin)) {
            code = W.run(I.dt, nacc, nrej);
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const int i = lane + G * r;
                if (i < nS) I.Y[(int64_t)i * I.ldY + c] = W.y[r];
                else if (i == nS && EN) I.T[c] = W.y[r];
            }
        }
        if (lane == 0) {
            if (I.status) I.status[c] = (uint8_t)code;
            if (I.stats) {
                int32_t* st = I.stats + KIN_NSTATS * c;
                st[0] = W.nfe;
                st[1] = nacc;
                st[2] = nrej;
                st[3] = 0;
                st[4] = 0;
            }
        }
    }
}

inline int rkck_group(int nV) { return warp_cell_lanes(KIN_RKCK, nV); }

template <typename R, bool EN>
inline size_t group_smem_bytes(const MechDev& M, int threads, int G)
{
    return (size_t)warp_group_words<R, EN>(M) * (threads / G) * 8;
}

template <typename R, int NR, bool EN, int G>
inline cudaError_t warp_rkck_launch_nr(Launch& L, int blocks, int threads, cudaStream_t st)
{
    const size_t sm = group_smem_bytes<R, EN>(L.M, threads, G);
    cudaError_t e = cudaFuncSetAttribute(warp_rkck_kernel<R, NR, EN, G>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    warp_rkck_kernel<R, NR, EN, G><<<blocks, threads, sm, st>>>(L);
    return cudaGetLastError();
}

template <typename R, int NR, bool EN, int G>
inline cudaError_t warp_rkck_occ_nr(const MechDev& M, int threads, int* bps)
{
    const size_t sm = group_smem_bytes<R, EN>(M, threads, G);
    cudaError_t e = cudaFuncSetAttribute(warp_rkck_kernel<R, NR, EN, G>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, warp_rkck_kernel<R, NR, EN, G>, threads, sm);
}

template <typename R, int NR, int OCC, bool EN>
inline cudaError_t warp_launch_nr(Launch& L, int blocks, int threads, cudaStream_t st)
{
    const size_t sm = warp_smem_bytes<R, EN>(L.M, threads);
    cudaError_t e = cudaFuncSetAttribute(warp_init_kernel<R, NR, OCC, EN>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(warp_integrate_kernel<R, NR, OCC, EN>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    warp_init_kernel<R, NR, OCC, EN><<<blocks, threads, sm, st>>>(L);
    e = launch_sort(L, st);
    if (e != cudaSuccess) return e;
    warp_integrate_kernel<R, NR, OCC, EN><<<blocks, threads, sm, st>>>(L);
    return cudaGetLastError();
}

template <typename R, int NR, int OCC, bool EN>
inline cudaError_t warp_occ_nr(const MechDev& M, int precision, int threads, int* bps)
{
    const size_t sm = warp_smem_bytes<R, EN>(M, threads);
    cudaError_t e = cudaFuncSetAttribute(warp_integrate_kernel<R, NR, OCC, EN>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, warp_integrate_kernel<R, NR, OCC, EN>,
                                                         threads, sm);
}

// Register-vector width for a state of n components (component l + 32 r, r < NR).
__host__ __device__ inline int warp_nr(int n) { return n <= 32 ? 1 : n <= 64 ? 2 : n <= 128 ? 4 : 8; }

template <typename R, int OCC, bool EN>
inline cudaError_t warp_launch(Launch& L, int blocks, int threads, cudaStream_t st)
{
    switch (warp_nr(L.nV)) {
    case 1: return warp_launch_nr<R, 1, OCC, EN>(L, blocks, threads, st);
    case 2: return warp_launch_nr<R, 2, OCC, EN>(L, blocks, threads, st);
    case 4: return warp_launch_nr<R, 4, OCC, EN>(L, blocks, threads, st);
    default: return warp_launch_nr<R, 8, OCC, EN>(L, blocks, threads, st);
    }
}

template <typename R, int OCC, bool EN>
inline cudaError_t warp_occ(const MechDev& M, int nV, int precision, int threads, int* bps)
{
    switch (warp_nr(nV)) {
    case 1: return warp_occ_nr<R, 1, OCC, EN>(M, precision, threads, bps);
    case 2: return warp_occ_nr<R, 2, OCC, EN>(M, precision, threads, bps);
    case 4: return warp_occ_nr<R, 4, OCC, EN>(M, precision, threads, bps);
    default: return warp_occ_nr<R, 8, OCC, EN>(M, precision, threads, bps);
    }
}

template <typename R, bool EN>
inline cudaError_t warp_rkck_launch(Launch& L, int blocks, int threads, cudaStream_t st)
{
    if (rkck_group(L.nV) == 16) return warp_rkck_launch_nr<R, 1, EN, 16>(L, blocks, threads, st);
    switch (warp_nr(L.nV)) {
    case 1: return warp_rkck_launch_nr<R, 1, EN, 32>(L, blocks, threads, st);
    case 2: return warp_rkck_launch_nr<R, 2, EN, 32>(L, blocks, threads, st);
    case 4: return warp_rkck_launch_nr<R, 4, EN, 32>(L, blocks, threads, st);
    default: return warp_rkck_launch_nr<R, 8, EN, 32>(L, blocks, threads, st);
    }
}

template <typename R, bool EN>
inline cudaError_t warp_rkck_occ(const MechDev& M, int nV, int precision, int threads, int* bps)
{
    (void)precision;
    if (rkck_group(nV) == 16) return warp_rkck_occ_nr<R, 1, EN, 16>(M, threads, bps);
    switch (warp_nr(nV)) {
    case 1: return warp_rkck_occ_nr<R, 1, EN, 32>(M, threads, bps);
    case 2: return warp_rkck_occ_nr<R, 2, EN, 32>(M, threads, bps);
    case 4: return warp_rkck_occ_nr<R, 4, EN, 32>(M, threads, bps);
    default: return warp_rkck_occ_nr<R, 8, EN, 32>(M, threads, bps);
    }
}

}  // namespace kin
