// kernels.cuh -- sm_103a kernels of the batched kinetics integrator (templates;
// instantiated per method and precision in inst_*.cu).
//
// Design (one GB300; FP64 runs at 1/64 of the FP32 rate, so the FP64 pipe,
// not HBM, bounds this path):
//  * One lane integrates one cell, as in the paper's thread-per-ODE design
//    (Section 3), but each loop iteration of a lane performs exactly ONE
//    evaluation of f. The method's control flow (RKCK stages, RKC stages,
//    finite-difference Jacobian columns, accept/reject) is a per-lane state
//    machine around that single call, so lanes of a warp in different phases
//    or on cells with different stage counts still execute f together;
//    divergence costs only the per-phase bookkeeping.
//  * A uniform pre-pass (init_kernel) does, for every cell and in lockstep
//    across the warp, the work every cell needs before its first step: the
//    rate constants (T is fixed over the flow step), f(y0), and for RKC the
//    Gershgorin spectral radius and the initial step of Section 2.3. The
//    initial step predicts a cell's cost (steps ~ dt/h1), so cells are bucket
//    sorted longest-first before the main kernel: longest-processing-time
//    order keeps the persistent grid's tail short.
//  * The main kernel is persistent: lanes pull cells from a warp-aggregated
//    atomic queue in that order and a lane that finishes its cell takes the
//    next one immediately.
//  * Working arrays are element-major in the workspace (coalesced per warp).
//  * f (Section 2.1): concentrations from the ideal gas law, Omega_j from the
//    stored rate constants, third-body and Lindemann falloff factors, and the
//    stoichiometric sum as a gather over a species-major CSR of net
//    coefficients (no scattered read-modify-write). Template parameter R is
//    the rate arithmetic type: double, or float for the mixed-precision path
//    (state, stage accumulation, norm and control stay double).
//  * No tensor cores: the stoichiometric contraction is sparse (about four
//    nonzeros per reaction).
//  * Code size: the integrator's loops over the state vector are not
//    unrolled (#pragma unroll 1) and the FP64 division, square root and power
//    are called out of line. A lane kernel holds every phase of the method,
//    and unrolled copies of some thirty short loops had made it 150 KB of
//    instructions; a smaller kernel waits less on instruction fetch (13
//    species: 2.105 M against 2.093 M cells/s).
#pragma once
#ifndef __CUDACC_RTC__  // run-time compilation (generated f) brings its own definitions
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#endif

#include "kin_dev.cuh"

namespace kin {

// IEEE FP64 division and square root, and the FP64 power, kept out of line:
// each library sequence is 2-9 KB of code, and one copy per kernel instead
// of one per use keeps the hot loops' instructions in cache (the warp
// layout's per-cell control has a dozen such uses). Same results as inline.
static __device__ __noinline__ double ddiv(double a, double b) { return a / b; }
static __device__ __noinline__ double dsqrt(double a) { return sqrt(a); }
static __device__ __noinline__ double dpow(double a, double b) { return pow(a, b); }
// a / b in the rate type: the FP64 division out of line, FP32 inline.
template <typename R>
__device__ __forceinline__ R rdiv(R a, R b)
{
    if constexpr (sizeof(R) == 8) return ddiv(a, b);
    else return a / b;
}


// ---------------------------------------------------------------- helpers --
template <typename T>
struct Lane {
    T* p;
    int32_t s;  // stride between elements (lanes or cells, < 2^31)
    __device__ __forceinline__ T& operator[](int i) const { return p[(int64_t)i * s]; }
};

template <typename R>
struct Tab;
template <>
struct Tab<double> {
    __device__ static const double* invW(const MechDev& M) { return M.invW; }
    __device__ static const double* eff(const MechDev& M) { return M.eff; }
    __device__ static const double* nu(const MechDev& M) { return M.csr_nu; }
    __device__ static const double* nuW(const MechDev& M) { return M.csr_nuW; }
    __device__ static double ex(double a) { return exp(a); }
    __device__ static double inv(double a);
    static constexpr double sqrt_u = 1.4901161193847656e-08;  // sqrt(2^-52)
};
template <>
struct Tab<float> {
    __device__ static const float* invW(const MechDev& M) { return M.invW32; }
    __device__ static const float* eff(const MechDev& M) { return M.eff32; }
    __device__ static const float* nu(const MechDev& M) { return M.csr_nu32; }
    __device__ static const float* nuW(const MechDev& M) { return M.csr_nuW32; }
    __device__ static float inv(float a) { return 1.0f / a; }
    // exp in FP32 after an exact split a = n ln2 + r formed in FP64, so the
    // FP32 rounding of a large exponent (|a| ~ 40) does not cost 2e-6
    // relative accuracy: k = 2^n expf(r) with |r| <= ln2/2.
    __device__ static float ex(double a)
    {
        const double n = rint(a * 1.4426950408889634);
        const float r = (float)fma(-n, 0.6931471805599453, a);
        return ldexpf(expf(r), (int)n);
    }
    static constexpr double sqrt_u = 3.4526698300124393e-04;  // sqrt(2^-23)
};

// Rate constants of one cell (Eq. (E:rxn-const)); T is fixed for the call.
// K_j = exp(ln A_j + beta_j ln T - (Ea_j/R)/T); for falloff reactions
// KR_fo = k_0/k_inf. The exponent is formed in double; the exp runs in R.
template <typename R>
__device__ void rate_constants(const MechDev& M, double T, Lane<R> K, Lane<R> KR)
{
    const double lnT = log(T), invT = ddiv(1.0, T);
    for (int j = 0; j < M.nR; ++j) {
        const double a = M.lnA[j] + M.beta[j] * lnT - M.EaR[j] * invT;
        K[j] = Tab<R>::ex(a);
        const int fo = M.rxn[j].fo;
        if (fo >= 0) {
            const double a0 = M.lnA0[j] + M.beta0[j] * lnT - M.Ea0R[j] * invT;
            KR[fo] = Tab<R>::ex(a0 - a);
        }
    }
}

// f(x) -> out (Eqs. (E:mass), (E:spec-rate), (E:rxn-rate)). Ctot = p/(R T) in
// mol/cm^3, invCtot its inverse. C and OM are lane scratch (nS and nR). R is
// the arithmetic type; the rate constants K, KR are stored in KT (float
// constants promoted to double when the mixed-precision path evaluates f in
// FP64 for its spectral-radius estimate).
template <typename R, typename KT>
__device__ void feval(const MechDev& M, double Ctot, double invCtot, Lane<KT> K, Lane<KT> KR,
                      Lane<R> C, Lane<R> OM, Lane<double> x, Lane<double> out)
{
    const int nS = M.nS, nR = M.nR;
    const R* __restrict__ invW = Tab<R>::invW(M);
    // mixture: S = sum Y/W = 1/Wbar, rho = Ctot Wbar, C_k = rho Y_k / W_k
    // (two partial sums per reduction: shorter dependent chains on the FP64 pipe)
    R S0 = R(0), S1 = R(0);
    int i = 0;
    for (; i + 1 < nS; i += 2) {
        const R m0 = (R)x[i] * invW[i];
        const R m1 = (R)x[i + 1] * invW[i + 1];
        C[i] = m0;
        C[i + 1] = m1;
        S0 += m0;
        S1 += m1;
    }
    if (i < nS) {
        const R m0 = (R)x[i] * invW[i];
        C[i] = m0;
        S0 += m0;
    }
    const R S = S0 + S1;
    const R rho = (R)Ctot * Tab<R>::inv(S);
    for (int k = 0; k < nS; ++k) C[k] = C[k] * rho;
    // rates of progress
    const R* __restrict__ eff = Tab<R>::eff(M);
    for (int j = 0; j < nR; ++j) {
        const Rxn r = M.rxn[j];
        R q = (R)K[j];
        if (r.r0 >= 0) q *= C[r.r0];
        if (r.r1 >= 0) q *= C[r.r1];
        if (r.type != KIN_RXN_PLAIN) {
            const R* a = eff + (int64_t)r.row * nS;
            R M0 = R(0), M1 = R(0);
            int k = 0;
            for (; k + 1 < nS; k += 2) {
                M0 += a[k] * C[k];
                M1 += a[k + 1] * C[k + 1];
            }
            if (k < nS) M0 += a[k] * C[k];
            const R Mc = M0 + M1;
            if (r.type == KIN_RXN_THIRD_BODY) {
                q *= Mc;
            } else {
                const R Pr = (R)KR[r.fo] * Mc;
                q *= rdiv<R>(Pr, R(1) + Pr);
            }
        }
        OM[j] = q;
    }
    // W_i omega_i = sum_j (W_i nu_ij) Omega_j (gather over the species' row,
    // W_i folded into its coefficients); dY_i/dt = W_i omega_i / rho
    const R* __restrict__ nuW = Tab<R>::nuW(M);
    const double invrho = (double)S * invCtot;
    for (int sp = 0; sp < nS; ++sp) {
        R w0 = R(0), w1 = R(0);
        const int e1 = M.csr_ptr[sp + 1];
        int e = M.csr_ptr[sp];
        for (; e + 1 < e1; e += 2) {
            w0 += nuW[e] * OM[M.csr_rxn[e]];
            w1 += nuW[e + 1] * OM[M.csr_rxn[e + 1]];
        }
        if (e < e1) w0 += nuW[e] * OM[M.csr_rxn[e]];
        out[sp] = (double)(w0 + w1) * invrho;
    }
}

// f with the energy equation (Eqs. (E:mass), (E:energy)): x = {Y_1..Y_nS, T}.
// The rate constants (Eq. (E:rxn-const)), the density and the concentrations
// follow the state's own T at every evaluation; the enthalpy sum
// sum_i H_i(T) omega_i and the mixture heat capacity cp = sum_i Y_i cp_i/W_i
// are FP64. dT/dt = -(sum_i H_i omega_i) / (rho cp), H_i = Hf_i + cp_i (T - T_REF).
template <typename R>
__device__ void feval_energy(const MechDev& M, double p, Lane<R> C, Lane<R> OM, Lane<double> x,
                             Lane<double> out)
{
    const int nS = M.nS, nR = M.nR;
    const double T = x[nS];
    const double lnT = log(T), invT = ddiv(1.0, T);
    const double Ctot = p * 1e-6 * invT * (1.0 / R_GAS), invCtot = ddiv(1.0, Ctot);
    const R* __restrict__ invW = Tab<R>::invW(M);
    R S0 = R(0), S1 = R(0);
    int i = 0;
    for (; i + 1 < nS; i += 2) {
        const R m0 = (R)x[i] * invW[i];
        const R m1 = (R)x[i + 1] * invW[i + 1];
        C[i] = m0;
        C[i + 1] = m1;
        S0 += m0;
        S1 += m1;
    }
    if (i < nS) {
        const R m0 = (R)x[i] * invW[i];
        C[i] = m0;
        S0 += m0;
    }
    const R S = S0 + S1;
    const R rho = (R)Ctot * Tab<R>::inv(S);
    for (int k = 0; k < nS; ++k) C[k] = C[k] * rho;
    const R* __restrict__ eff = Tab<R>::eff(M);
    for (int j = 0; j < nR; ++j) {
        const Rxn r = M.rxn[j];
        const double a = M.lnA[j] + M.beta[j] * lnT - M.EaR[j] * invT;
        R q = Tab<R>::ex(a);
        if (r.r0 >= 0) q *= C[r.r0];
        if (r.r1 >= 0) q *= C[r.r1];
        if (r.type != KIN_RXN_PLAIN) {
            const R* a_ = eff + (int64_t)r.row * nS;
            R M0 = R(0), M1 = R(0);
            int k = 0;
            for (; k + 1 < nS; k += 2) {
                M0 += a_[k] * C[k];
                M1 += a_[k + 1] * C[k + 1];
            }
            if (k < nS) M0 += a_[k] * C[k];
            const R Mc = M0 + M1;
            if (r.type == KIN_RXN_THIRD_BODY) {
                q *= Mc;
            } else {
                const double a0 = M.lnA0[j] + M.beta0[j] * lnT - M.Ea0R[j] * invT;
                const R Pr = Tab<R>::ex(a0 - a) * Mc;
                q *= rdiv<R>(Pr, R(1) + Pr);
            }
        }
        OM[j] = q;
    }
    const R* __restrict__ nu = Tab<R>::nu(M);
    const double invrho = (double)S * invCtot;
    const double dT = T - T_REF;
    double hw = 0.0, cpm = 0.0;
    for (int sp = 0; sp < nS; ++sp) {
        R w0 = R(0), w1 = R(0);
        const int e1 = M.csr_ptr[sp + 1];
        int e = M.csr_ptr[sp];
        for (; e + 1 < e1; e += 2) {
            w0 += nu[e] * OM[M.csr_rxn[e]];
            w1 += nu[e + 1] * OM[M.csr_rxn[e + 1]];
        }
        if (e < e1) w0 += nu[e] * OM[M.csr_rxn[e]];
        const double om = (double)(w0 + w1);
        out[sp] = om * (M.W[sp] * invrho);
        hw += (M.Hf[sp] + M.cp[sp] * dT) * om;
        cpm += x[sp] * M.cpW[sp];
    }
    out[nS] = ddiv(-hw * invrho, cpm);
}

__device__ __forceinline__ int find_inst(const Launch& L, long long g)
{
    int lo = 0, hi = L.n_inst - 1;
    while (lo < hi) {  // largest i with start[i] <= g
        const int mid = (lo + hi + 1) >> 1;
        if (L.start[mid] <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Warp-aggregated pop of the next queue position for every active lane.
__device__ __forceinline__ long long pop_cell(unsigned long long* q)
{
    const unsigned mask = __activemask();
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    const int rank = __popc(mask & ((1u << lane) - 1u));
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(q, (unsigned long long)__popc(mask));
    base = __shfl_sync(mask, base, leader);
    return (long long)(base + rank);
}

// Vector slots of a lane's working set.
enum Vec : int { V_Y = 0, V_F0, V_A, V_B, V_C, V_X, V_FX, V_RS };
// RKCK reuses slots: F[1..5] = V_A, V_B, V_C, V_FX, V_RS; the stage point is V_X.

extern __shared__ __align__(16) unsigned char kin_smem[];

// Per-lane views of the workspace. Staging level STG places the arrays f
// touches most in shared memory, element-major across the block
// ([element][thread]): 1 = concentrations and rates of progress, 2 = also
// the cell's rate constants. Otherwise they live in the lane's slice of the
// workspace ([element][lane]): C [nS], Omega [nR], k [nR], k0/kinf [nFO].
template <typename R, int STG>
struct Views {
    const Launch& L;
    const MechDev& M;
    int64_t slot;
    Lane<R> C, OM, Kl, KRl;
    Lane<double> C64, OM64;  // mixed precision: FP64 scratch of the spectral-radius f
    double* vbase;
    __device__ Views(const Launch& l, int64_t sl) : L(l), M(l.M), slot(sl)
    {
        R* rb = reinterpret_cast<R*>(L.lane_r) + sl;
        const int64_t ns = L.nslots;
        R* sb = reinterpret_cast<R*>(kin_smem) + threadIdx.x;
        const int64_t bs = blockDim.x;
        if (STG >= 1) {
            C = Lane<R>{sb, (int32_t)bs};
            OM = Lane<R>{sb + (int64_t)M.nS * bs, (int32_t)bs};
        } else {
            C = Lane<R>{rb, (int32_t)ns};
            OM = Lane<R>{rb + (int64_t)M.nS * ns, (int32_t)ns};
        }
        if (STG >= 2) {
            Kl = Lane<R>{sb + (int64_t)(M.nS + M.nR) * bs, (int32_t)bs};
            KRl = Lane<R>{sb + (int64_t)(M.nS + 2 * M.nR) * bs, (int32_t)bs};
        } else {
            Kl = Lane<R>{rb + (int64_t)(M.nS + M.nR) * ns, (int32_t)ns};
            KRl = Lane<R>{rb + (int64_t)(M.nS + 2 * M.nR) * ns, (int32_t)ns};
        }
        vbase = L.vec + sl;
        C64 = Lane<double>{L.lane_sig + sl, (int32_t)ns};
        OM64 = Lane<double>{L.lane_sig + (int64_t)M.nS * ns + sl, (int32_t)ns};
    }
    __device__ __forceinline__ Lane<double> V(int v) const
    {
        return Lane<double>{vbase + (int64_t)v * L.nV * L.nslots, (int32_t)L.nslots};
    }
    __device__ __forceinline__ Lane<R> K(int64_t g) const
    {
        return Lane<R>{reinterpret_cast<R*>(L.cell_k) + g, (int32_t)L.total};
    }
    __device__ __forceinline__ Lane<R> KR(int64_t g) const
    {
        return Lane<R>{reinterpret_cast<R*>(L.cell_k) + (int64_t)M.nR * L.total + g, (int32_t)L.total};
    }
    __device__ __forceinline__ Lane<double> EVcell(int64_t g) const
    {
        return Lane<double>{L.cell_ev + g, (int32_t)L.total};
    }
    __device__ __forceinline__ Lane<double> F0cell(int64_t g) const
    {
        return Lane<double>{L.cell_f0 + g, (int32_t)L.total};
    }
};

// Weighted RMS norm, Eq. (E:rmsE), of d with T_i = atol + rtol max(|a|,|b|).
__device__ __forceinline__ double rms(int n, double rtol, double atol, Lane<double> d,
                                      Lane<double> a, Lane<double> b)
{
    double acc = 0.0;
#pragma unroll 1
    for (int i = 0; i < n; ++i) {
        const double sc = atol + rtol * fmax(fabs(a[i]), fabs(b[i]));
        const double r = ddiv(d[i], sc);
        acc += r * r;
    }
    return dsqrt(ddiv(acc, (double)n));
}

// ------------------------------------------------- power-method sigma ---
// Nonlinear power method (the paper's spectral-radius estimator, end of
// Section 2.3): w = f(y + v) - f(y) ~ J v with v rescaled to length
// dyn = sqrt(u) ||y||_2, warm-started from the previous estimate's direction
// (f(y0) at the first estimate, all ones if that is zero); stop when two
// successive ||w||/dyn agree to 1 % or after 20 products; sigma = 1.2 x the
// last value (the iteration approaches |lambda_max| from below).
// Spectral-radius estimates evaluate f in FP64 in both precisions (u = 2^-52):
// with FP32 rate arithmetic the rounding noise of f(y + v) - f(y) can exceed
// the difference itself, and the iteration would neither converge nor agree
// with the FP64 estimate.
constexpr double SIG_SQRT_U = 1.4901161193847656e-08;  // sqrt(2^-52)

// ------------------------------------------ Newton-refined FP64 helpers ---
// The per-lane step control runs on the FP64 pipe while the other lanes of
// the warp wait, so its FP64 instruction count matters. These helpers take a
// low-precision seed (the approximate FP64 reciprocal instruction, the FP32
// cube root or power) and refine it with one Newton-Raphson step in FP64,
// which squares the seed's relative error (reciprocal: below 2^-19.9, measured
// over 4M log-uniform inputs on GB300 -> ~1e-12 after the step): enough for an
// error norm and a step-size factor, which only need to reproduce the FP64
// decisions. Outside the FP32 normal range the plain FP64 operation is used.
__device__ __forceinline__ bool f32_normal(double x)
{
    const int e = (__double2hiint(x) >> 20) & 0x7ff;  // biased exponent (sign ignored)
    return e > 1023 - 120 && e < 1023 + 120;
}

// 1/x: Newton r1 = r0 + r0 (1 - x r0) from rcp.approx.ftz.f64 (no FP32
// round trip, so no conversions on the FP64 pipe).
__device__ __forceinline__ double rcp_newton(double x)
{
    if (!f32_normal(x)) return ddiv(1.0, x);
    double r0;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r0) : "d"(x));
    return fma(r0, fma(-x, r0, 1.0), r0);
}

// a^(1/3) for a > 0: Newton c1 = c0 - (c0^3 - a) / (3 c0^2) = c0 + (a / c0^2 - c0) / 3.
__device__ __forceinline__ double cbrt_newton(double a)
{
    if (!f32_normal(a)) return cbrt(a);
    const double c0 = (double)cbrtf((float)a);
    return c0 + (a * rcp_newton(c0 * c0) - c0) * (1.0 / 3.0);
}

// x^(-1/5) and x^(-1/4) for x > 0, the RKCK step-size factors: Newton on
// y^(-p) = x, y1 = y0 + y0 (1 - x y0^p) / p, from y0 = powf(x, -1/p). A seed
// error e becomes (p + 1)/2 e^2 (powf is within 4 ulp: below 5e-12 after the
// step, ample for a step-size factor).
__device__ __forceinline__ double rpow5_newton(double x)
{
    if (!f32_normal(x)) return dpow(x, -0.2);
    const double y0 = (double)powf((float)x, -0.2f);
    const double y2 = y0 * y0;
    const double u = fma(-(x * y0), y2 * y2, 1.0);
    return fma(y0 * u, 0.2, y0);
}

// x^(-1/6) for x > 0: the RKC controller's err^(-1/3) from x = err^2.
__device__ __forceinline__ double rpow6_newton(double x)
{
    if (!f32_normal(x)) return dpow(x, -1.0 / 6.0);
    const double y0 = (double)powf((float)x, -1.0f / 6.0f);
    const double y2 = y0 * y0;
    const double u = fma(-(x * y2), y2 * y2, 1.0);
    return fma(y0 * u, 1.0 / 6.0, y0);
}

__device__ __forceinline__ double rpow4_newton(double x)
{
    if (!f32_normal(x)) return dpow(x, -0.25);
    const double y0 = (double)powf((float)x, -0.25f);
    const double y2 = y0 * y0;
    const double u = fma(-(x * y2), y2, 1.0);
    return fma(y0 * u, 0.25, y0);
}
// 1/x in the FP64 evaluation of f (the mixture density): a second Newton
// step on rcp_newton takes the error from ~1e-12 to rounding level, so f
// stays an FP64-accurate function of the state.
__device__ __forceinline__ double Tab<double>::inv(double a)
{
    const double r = rcp_newton(a);
    return fma(r, fma(-a, r, 1.0), r);
}

struct PowerState {
    int k;
    double prev, dyn, sig;
};

__device__ __forceinline__ void power_begin(int nS, Lane<double> Y, Lane<double> EV, Lane<double> X,
                                            PowerState& P)
{
    double yn = 0.0, vn = 0.0;
#pragma unroll 1
    for (int i = 0; i < nS; ++i) {
        yn += Y[i] * Y[i];
        vn += EV[i] * EV[i];
    }
    yn = dsqrt(yn);
    P.dyn = yn > 0.0 ? SIG_SQRT_U * yn : SIG_SQRT_U;
    vn = dsqrt(vn);
    if (!(vn > 0.0) || !isfinite(vn)) {
#pragma unroll 1
        for (int i = 0; i < nS; ++i) EV[i] = 1.0;
        vn = dsqrt((double)nS);
    }
    const double sc = ddiv(P.dyn, vn);
#pragma unroll 1
    for (int i = 0; i < nS; ++i) {
        EV[i] = EV[i] * sc;
        X[i] = Y[i] + EV[i];
    }
    P.k = 1;
    P.prev = 0.0;
    P.sig = 0.0;
}

// FX holds f(Y + EV), F0 = f(Y) (both FP64). Updates EV; returns true when
// the estimate is final (then sigma = 1.2 P.sig); otherwise X is set to the
// next point Y + EV.
__device__ __forceinline__ bool power_post(int nS, Lane<double> Y, Lane<double> F0, Lane<double> EV,
                           Lane<double> X, Lane<double> FX, PowerState& P)
{
    double wn = 0.0;
#pragma unroll 1
    for (int i = 0; i < nS; ++i) {
        const double w = FX[i] - F0[i];
        FX[i] = w;
        wn += w * w;
    }
    wn = dsqrt(wn);
    P.sig = ddiv(wn, P.dyn);
    if (!(wn > 0.0) || !isfinite(wn)) return true;
    const double sc = ddiv(P.dyn, wn);
#pragma unroll 1
    for (int i = 0; i < nS; ++i) EV[i] = FX[i] * sc;
    if (P.k >= 2 && fabs(P.sig - P.prev) <= 0.01 * P.sig) return true;
    P.prev = P.sig;
    if (++P.k > 20) return true;
#pragma unroll 1
    for (int i = 0; i < nS; ++i) X[i] = Y[i] + EV[i];
    return false;
}

// How the lane kernels evaluate the isothermal f: a policy class F with
// F::eval<R, KT>(M, Ctot, invCtot, K, KR, C, OM, x, out). TableF is feval
// over the mechanism's device tables (any mechanism, either precision); a
// generated policy (FP64 only) is f for one mechanism as straight-line code,
// compiled at run time, with the same arguments.
struct TableF {
    template <typename R, typename KT>
    __device__ __forceinline__ static void eval(const MechDev& M, double Ctot, double invCtot, Lane<KT> K,
                                                Lane<KT> KR, Lane<R> C, Lane<R> OM, Lane<double> x,
                                                Lane<double> out)
    {
        feval<R, KT>(M, Ctot, invCtot, K, KR, C, OM, x, out);
    }
    // f with the energy equation (x = {Y, T})
    template <typename R>
    __device__ __forceinline__ static void eval_energy(const MechDev& M, double p, Lane<R> C, Lane<R> OM,
                                                       Lane<double> x, Lane<double> out)
    {
        feval_energy<R>(M, p, C, OM, x, out);
    }
};

// f in FP64 for a spectral-radius estimate: the lane's rate scratch in the
// FP64 path, the separate FP64 scratch in the mixed-precision path (whose
// rate constants are the same FP32 values, promoted).
template <typename R, int STG, typename F>
__device__ __forceinline__ void feval_sig(const Views<R, STG>& W, double Ctot, double invCtot,
                                          Lane<R> K, Lane<R> KR, Lane<double> x, Lane<double> out)
{
    if constexpr (sizeof(R) == 4)
        F::template eval<double, R>(W.M, Ctot, invCtot, K, KR, W.C64, W.OM64, x, out);
    else
        F::template eval<double, R>(W.M, Ctot, invCtot, K, KR, W.C, W.OM, x, out);
}

// ------------------------------------------------------------- pre-pass --
// For every cell g (grid-stride, uniform across lanes): rate constants, f(y0),
// and for RKC the spectral radius (Section 2.3) and the initial step
// h1 = 0.1 h0 / ||Delta_0||^(1/2), h0 = 1/sigma.
template <int METHOD, typename R, int STG, bool EN, typename F = TableF>
__global__ void __launch_bounds__(128) init_kernel(const __grid_constant__ Launch L)
{
    const int64_t slot = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (slot >= L.nslots) return;
    Views<R, STG> W(L, slot);
    const MechDev& M = L.M;
    const int nS = M.nS, n = L.nV;
    for (int64_t g = slot; g < L.total; g += L.nslots) {
        const int ii = find_inst(L, g);
        const InstDev& I = L.inst[ii];
        const int64_t c = g - L.start[ii];
        const double T = I.T[c], p = I.p[c];
        const double Ctot = ddiv(p * 1e-6, R_GAS * T), invCtot = ddiv(1.0, Ctot);
        Lane<R> K = W.K(g), KR = W.KR(g);
        if constexpr (!EN) rate_constants<R>(M, T, K, KR);
        // f in the rate type, and f in FP64 for the spectral radius
        auto frate = [&](Lane<double> x, Lane<double> o) {
            if constexpr (EN) F::template eval_energy<R>(M, p, W.C, W.OM, x, o);
            else F::template eval<R, R>(M, Ctot, invCtot, K, KR, W.C, W.OM, x, o);
        };
        auto fsig = [&](Lane<double> x, Lane<double> o) {
            if constexpr (EN) {
                if constexpr (sizeof(R) == 4) F::template eval_energy<double>(M, p, W.C64, W.OM64, x, o);
                else F::template eval_energy<double>(M, p, W.C, W.OM, x, o);
            } else {
                feval_sig<R, STG, F>(W, Ctot, invCtot, K, KR, x, o);
            }
        };
        Lane<double> Y = W.V(V_Y), F0 = W.F0cell(g), X = W.V(V_X), FX = W.V(V_FX), RS = W.V(V_RS);
        bool ok = true;
#pragma unroll 1
        for (int i = 0; i < n; ++i) {
            const double y = i < nS ? I.Y[(int64_t)i * I.ldY + c] : T;
            Y[i] = y;
            X[i] = y;
            RS[i] = 0.0;
        }
        frate(Y, F0);
#pragma unroll 1
        for (int i = 0; i < n; ++i) ok &= isfinite(F0[i]);
        uint8_t st = ok ? 0 : KIN_CELL_NONFINITE;
        double sigma = 0.0, h = I.dt;
        int nfe = 1, nfs = 0;  // f evaluations, and those inside the sigma estimate
        // base point of the FP64 spectral-radius differences: f(y0) itself in
        // FP64, its FP64 re-evaluation in the mixed-precision path
        Lane<double> B = F0;
        if (METHOD == KIN_RKC && ok && sizeof(R) == 4) {
            B = W.V(V_B);
            fsig(Y, B);
            nfe++;
            nfs++;
        }
        if (METHOD == KIN_RKC && ok && L.sigma_method == KIN_SIGMA_POWER) {
            Lane<double> EV = W.EVcell(g);
#pragma unroll 1
            for (int i = 0; i < n; ++i) EV[i] = B[i];  // first direction: f(y0)
            PowerState P;
            power_begin(n, Y, EV, X, P);
            for (;;) {
                fsig(X, FX);
                nfe++;
                nfs++;
                if (power_post(n, Y, B, EV, X, FX, P)) break;
            }
            sigma = 1.2 * P.sig;
        } else if (METHOD == KIN_RKC && ok) {
#pragma unroll 1
            for (int k = 0; k < n; ++k) {  // Gershgorin columns
                const double eps = SIG_SQRT_U * fmax(fabs(Y[k]), I.atol);
                X[k] = Y[k] + eps;
                fsig(X, FX);
                const double ie = ddiv(1.0, eps);
#pragma unroll 1
                for (int i = 0; i < n; ++i) RS[i] += fabs((FX[i] - B[i]) * ie);
                X[k] = Y[k];
            }
#pragma unroll 1
            for (int i = 0; i < n; ++i) sigma = fmax(sigma, RS[i]);
            nfe += n;
            nfs += n;
        }
        if (METHOD == KIN_RKC && ok) {
            if (!isfinite(sigma)) {
                st = KIN_CELL_NONFINITE;
            } else {
                double h0 = sigma > 0.0 ? ddiv(1.0, sigma) : I.dt;
                if (h0 > I.dt) h0 = I.dt;
#pragma unroll 1
                for (int i = 0; i < n; ++i) X[i] = Y[i] + h0 * F0[i];
                frate(X, FX);
                nfe++;
#pragma unroll 1
                for (int i = 0; i < n; ++i) X[i] = h0 * (FX[i] - F0[i]);  // Delta_0
                const double e0 = rms(n, I.rtol, I.atol, X, Y, Y);
                if (!isfinite(e0)) h = 0.1 * h0;
                else h = e0 > 0.0 ? ddiv(0.1 * h0, dsqrt(e0)) : I.dt;
                if (h > I.dt) h = I.dt;
                if (h < 1e-20 * I.dt) st = KIN_CELL_HMIN;
            }
        }
        L.cell_sig[g] = sigma;
        L.cell_h[g] = h;
        L.cell_nfe[g] = nfe;
        L.cell_nfs[g] = nfs;
        L.cell_st[g] = st;
    }
}

// ----------------------------------------------- longest-first ordering --
// Predicted cost of a cell: steps ~ dt/h1 (RKC). Bucket b >= 1 grows with
// log2(1 + dt/h1) in quarter octaves; cells already finished go to bucket 0.
__device__ __forceinline__ int cost_bucket(const Launch& L, int64_t g)
{
    if (L.cell_st[g] != 0) return 0;
    const int ii = find_inst(L, g);
    const double r = ddiv(L.inst[ii].dt, L.cell_h[g]);
    const int b = 1 + (int)(4.0f * log2f(1.0f + (float)r));
    return b < 1 ? 1 : (b > NBUCKET - 1 ? NBUCKET - 1 : b);
}


// ------------------------------------------------------------ integrator --
enum Phase : int {
    PH_F0 = 0,   // RKCK: f at the current accepted state -> F0
    PH_SIGBASE,  // RKC, mixed precision: FP64 f(Y) -> V_B, the base of the sigma differences
    PH_SIG,      // RKC: f at Y + eps_k e_k (Gershgorin column k) -> FX
    PH_POW,      // RKC: f at Y + v (power-method product) -> FX
    PH_STAGE,    // RKC: f(w_{j-1}) -> FX, then w_j
    PH_FINAL,    // RKC: f(w_s) -> FX, error estimate and control
    PH_K,        // RKCK: f at a stage point -> F[st]
};

__constant__ double CK_B[6][5] = {
    {0, 0, 0, 0, 0},
    {1.0 / 5.0, 0, 0, 0, 0},
    {3.0 / 40.0, 9.0 / 40.0, 0, 0, 0},
    {3.0 / 10.0, -9.0 / 10.0, 6.0 / 5.0, 0, 0},
    {-11.0 / 54.0, 5.0 / 2.0, -70.0 / 27.0, 35.0 / 27.0, 0},
    {1631.0 / 55296.0, 175.0 / 512.0, 575.0 / 13824.0, 44275.0 / 110592.0, 253.0 / 4096.0}};
// fifth-order weights c_i and error weights c_i - c*_i (Table 1)
__constant__ double CK_C[6] = {37.0 / 378.0, 0.0, 250.0 / 621.0, 125.0 / 594.0, 0.0, 512.0 / 1771.0};
__constant__ double CK_E[6] = {37.0 / 378.0 - 2825.0 / 27648.0, 0.0, 250.0 / 621.0 - 18575.0 / 48384.0,
                               125.0 / 594.0 - 13525.0 / 55296.0, -277.0 / 14336.0,
                               512.0 / 1771.0 - 1.0 / 4.0};

__device__ __forceinline__ int ck_slot(int st)
{
    // F[0] lives in V_F0; F[1..5] in the slots listed above
    return st == 0 ? V_F0 : (st <= 3 ? V_A + st - 1 : (st == 4 ? V_FX : V_RS));
}

struct LaneState {
    long long g;     // global cell index
    long long cell;  // index within the instance
    int inst;
    int phase, st, j, s, col;
    int attempts, nacc, nrej, nsig, nfe, nfs;
    int since_sigma;
    bool last, last_rejected, have_prev, sigma_here;
    int iw1, iw2;  // RKC: slots of w_{j-1}, w_{j-2}
    double t, dt, h, hh, hprev, cprev, sigma, eps, rtol, atol, Ctot, invCtot, invN, p;
    int in_v, out_v;  // vectors read and written by the next f evaluation
    PowerState P;     // RKC power-method sigma in progress
};

template <int METHOD, typename R, int STG, bool EN, typename F = TableF>
struct Integrator {
    Views<R, STG> W;
    const Launch& L;
    const MechDev& M;
    Lane<R> K, KR;

    __device__ Integrator(const Launch& l, int64_t sl) : W(l, sl), L(l), M(l.M) {}
    __device__ __forceinline__ Lane<double> V(int v) const { return W.V(v); }

    // ---------------------------------------------------------- cell I/O --
    // Take the next cell; returns false when the queue is exhausted. A cell
    // whose fate the pre-pass already decided is finished here directly.
    __device__ bool load_next(LaneState& S)
    {
        for (;;) {
            const long long q = pop_cell(L.queue);
            if (q >= L.total) return false;
            const long long g = (METHOD == KIN_RKC) ? (long long)L.order[q] : q;
            const int i = find_inst(L, g);
            const InstDev& I = L.inst[i];
            S.g = g;
            S.inst = i;
            S.cell = g - L.start[i];
            S.attempts = S.nacc = S.nrej = 0;
            S.nsig = METHOD == KIN_RKC ? 1 : 0;
            S.nfe = L.cell_nfe[g];
            S.nfs = L.cell_nfs[g];
            const uint8_t pre = L.cell_st[g];
            if (pre != 0) {  // Y stays as given
                finish_stats(S, pre);
                continue;
            }
            const double T = I.T[S.cell], p = I.p[S.cell];
            S.p = p;
            S.Ctot = ddiv(p * 1e-6, R_GAS * T);
            S.invCtot = ddiv(1.0, S.Ctot);
            if constexpr (!EN) {
                // the cell's rate constants into the lane's (coalesced or shared) copy
                K = W.Kl;
                KR = W.KRl;
                const Lane<R> Kc = W.K(g), KRc = W.KR(g);
                for (int j = 0; j < M.nR; ++j) K[j] = Kc[j];
                for (int j = 0; j < M.nFO; ++j) KR[j] = KRc[j];
            }
            const int n = L.nV;
            Lane<double> Y = V(V_Y), F0 = V(V_F0), F0c = W.F0cell(g);
#pragma unroll 1
            for (int k = 0; k < n; ++k) {
                Y[k] = k < M.nS ? I.Y[(int64_t)k * I.ldY + S.cell] : T;
                F0[k] = F0c[k];
            }
            if (METHOD == KIN_RKC && L.sigma_method == KIN_SIGMA_POWER) {
                // the pre-pass estimate's direction warm-starts the next one
                Lane<double> EV = V(V_RS), EVc = W.EVcell(g);
#pragma unroll 1
                for (int k = 0; k < n; ++k) EV[k] = EVc[k];
            }
            S.dt = I.dt;
            S.rtol = I.rtol;
            S.atol = I.atol;
            S.invN = ddiv(1.0, (double)n);
            S.t = 0.0;
            S.h = L.cell_h[g];
            S.sigma = L.cell_sig[g];
            S.since_sigma = 0;
            S.last = false;
            S.last_rejected = false;
            S.have_prev = false;
            S.sigma_here = true;
            S.hprev = S.cprev = 0.0;
            const int code = METHOD == KIN_RKC ? rkc_begin_step(S) : rkck_begin_attempt(S);
            if (code < 0) return true;
            store(S, code);
        }
    }

    __device__ void finish_stats(const LaneState& S, int code)
    {
        const InstDev& I = L.inst[S.inst];
        if (I.status) I.status[S.cell] = (uint8_t)code;
        if (I.stats) {
            int32_t* st = I.stats + KIN_NSTATS * S.cell;
            st[0] = S.nfe;
            st[1] = S.nacc;
            st[2] = S.nrej;
            st[3] = S.nsig;
            st[4] = S.nfs;
        }
    }

    __device__ void store(const LaneState& S, int code)
    {
        const InstDev& I = L.inst[S.inst];
        Lane<double> Y = V(V_Y);
        for (int k = 0; k < M.nS; ++k) I.Y[(int64_t)k * I.ldY + S.cell] = Y[k];
        if constexpr (EN) I.T[S.cell] = Y[M.nS];
        finish_stats(S, code);
    }

    // Slot holding f(Y) in FP64 during a spectral-radius estimate.
    static constexpr int V_BASE = sizeof(R) == 4 ? V_B : V_F0;

    // Start a spectral-radius estimate at Y; the mixed-precision path first
    // re-evaluates f(Y) in FP64 (V_B is free: the stage vectors are formed
    // after the estimate).
    __device__ void sigma_begin(LaneState& S)
    {
        if (sizeof(R) == 4) {
            S.phase = PH_SIGBASE;
            S.in_v = V_Y;
            S.out_v = V_B;
            return;
        }
        sigma_start(S);
    }

    // Power method (X = Y + v) or Gershgorin (X = Y + eps_0 e_0, RS = 0).
    __device__ void sigma_start(LaneState& S)
    {
        if (L.sigma_method == KIN_SIGMA_POWER) {
            power_begin(L.nV, V(V_Y), V(V_RS), V(V_X), S.P);
            S.phase = PH_POW;
            S.in_v = V_X;
            S.out_v = V_FX;
            return;
        }
        Lane<double> Y = V(V_Y), X = V(V_X), RS = V(V_RS);
#pragma unroll 1
        for (int i = 0; i < L.nV; ++i) {
            X[i] = Y[i];
            RS[i] = 0.0;
        }
        S.col = 0;
        S.eps = SIG_SQRT_U * fmax(fabs(Y[0]), S.atol);
        X[0] = Y[0] + S.eps;
        S.phase = PH_SIG;
        S.in_v = V_X;
        S.out_v = V_FX;
    }

    // Post-processing of one Gershgorin column. Returns true when sigma is done.
    __device__ bool sigma_column(LaneState& S)
    {
        Lane<double> Y = V(V_Y), X = V(V_X), RS = V(V_RS), FX = V(V_FX), F0 = V(V_BASE);
        const double ie = rcp_newton(S.eps);
#pragma unroll 1
        for (int i = 0; i < L.nV; ++i) RS[i] += fabs((FX[i] - F0[i]) * ie);
        X[S.col] = Y[S.col];
        if (++S.col < L.nV) {
            S.eps = SIG_SQRT_U * fmax(fabs(Y[S.col]), S.atol);
            X[S.col] = Y[S.col] + S.eps;
            return false;
        }
        double sg = 0.0;
#pragma unroll 1
        for (int i = 0; i < L.nV; ++i) sg = fmax(sg, RS[i]);
        S.sigma = sg;
        S.nsig++;
        S.since_sigma = 0;
        S.sigma_here = true;
        return true;
    }

    // ------------------------------------------------------------- RKC ---
    __device__ const double* coef(int s, int j) const
    {
        return M.rkc + ((int64_t)s * RKC_TAB_S + j) * RKC_TAB_W;
    }

    // Choose the next attempt (or a spectral-radius refresh). Returns a
    // finish code >= 0 if the cell must stop, else -1.
    __device__ int rkc_begin_step(LaneState& S)
    {
        if (S.attempts >= L.max_steps) return KIN_CELL_MAXSTEPS;
        if (S.since_sigma >= 25 || (S.last_rejected && !S.sigma_here)) {
            sigma_begin(S);
            return -1;
        }
        double hh = S.h;
        S.last = false;
        if (hh >= S.dt - S.t) {
            hh = S.dt - S.t;
            S.last = true;
        }
        const double sr = floor(1.0 + dsqrt(1.0 + 1.54 * hh * S.sigma));
        int s;
        if (sr < 2.0) {
            s = 2;
        } else if (sr > (double)SMAX) {
            s = SMAX;
            hh = ddiv((SMAX - 1.0) * (SMAX - 1.0) - 1.0, 1.54 * S.sigma);
            S.last = false;
        } else {
            s = (int)sr;
        }
        S.hh = hh;
        S.s = s;
        // w_1 = y + mu~_1 h f_0 into slot A; w_0 = y stays in V_Y
        const double m1 = coef(s, 1)[2] * hh;
        Lane<double> Y = V(V_Y), F0 = V(V_F0), A = V(V_A);
#pragma unroll 1
        for (int i = 0; i < L.nV; ++i) A[i] = Y[i] + m1 * F0[i];
        S.iw1 = V_A;
        S.iw2 = V_Y;
        S.j = 2;
        S.phase = PH_STAGE;
        S.in_v = V_A;
        S.out_v = V_FX;
        return -1;
    }

    // Weighted RMS norm (Eq. (E:rmsE)) of the error vectors of the lanes in
    // the final phase, left in their free slot nw; returns the sum of squares
    // on those lanes. The per-element work (weight, reciprocal, scaling) of
    // all of them is spread over every lane that reaches this point with
    // them, so that a warp whose lanes end their steps at different times
    // runs it in ceil(k n / 32) rounds instead of n rounds with k lanes
    // active. Each final-phase lane then adds its own squares in element
    // order: the result is bit for bit that of the lane alone.
    __device__ double final_norm(const LaneState& S, bool fin, int nw)
    {
        const unsigned mask = __activemask();
        const unsigned fm = __ballot_sync(mask, fin);
        if (fm == 0u) return 0.0;
        const int lane = threadIdx.x & 31;
        const int n = L.nV;
        const int nact = __popc(mask);
        const int rank = __popc(mask & ((1u << lane) - 1u));
        const int items = __popc(fm) * n;
        const int64_t ns = L.nslots;
        const int64_t slot0 = W.slot - lane;  // the warp's lanes hold consecutive slots
        for (int base = 0; base < items; base += nact) {
            const int t = base + rank;
            const bool live = t < items;
            const int f = live ? t / n : 0;
            unsigned m = fm;  // the f-th finishing lane
            for (int c = 0; c < f; ++c) m &= m - 1u;
            const int A = __ffs(m) - 1;
            const int a_iw1 = __shfl_sync(mask, S.iw1, A);
            const int a_nw = __shfl_sync(mask, nw, A);
            const double a_atol = __shfl_sync(mask, S.atol, A);
            const double a_rtol = __shfl_sync(mask, S.rtol, A);
            if (live) {
                const int i = t - f * n;
                double* const va = L.vec + slot0 + A;
                const double y = va[((int64_t)V_Y * n + i) * ns];
                const double w1 = va[((int64_t)a_iw1 * n + i) * ns];
                double* const pd = va + ((int64_t)a_nw * n + i) * ns;
                const double sc = a_atol + a_rtol * fmax(fabs(y), fabs(w1));
                *pd = *pd * rcp_newton(sc);
            }
        }
        __syncwarp(mask);
        double acc = 0.0;
        if (fin) {
            Lane<double> D = V(nw);
#pragma unroll 1
            for (int i = 0; i < n; ++i) {
                const double r = D[i];
                acc += r * r;
            }
        }
        return acc;
    }

    __device__ int rkc_post(LaneState& S)
    {
        const bool fin = S.phase == PH_FINAL;
        const bool sf = S.phase == PH_STAGE || fin;
        int nw = 0;
        if (sf) {
            // One pass serves both phases, so that lanes of a warp in either
            // share it instead of running two loops in turn. FX = f(w_{j-1}):
            //   stage j: w_j = (1-mu-nu) y + mu w_{j-1} + nu w_{j-2}
            //                  + mu~ h f_{j-1} + gamma~ h f_0;
            //   final:   Delta = 0.8 (y - w_s) + 0.4 h (f_0 + f_s), the same
            //            five-term form (nu = 0), into the free slot for
            //            final_norm.
            double c0, mu, nu, mt, gt;
            if (fin) {
                c0 = 0.8;
                mu = -0.8;
                nu = 0.0;
                mt = gt = 0.4 * S.hh;
            } else {
                const double* c = coef(S.s, S.j);
                mu = c[0];
                nu = c[1];
                mt = c[2] * S.hh;
                gt = c[3] * S.hh;
                c0 = c[4];
            }
            nw = (S.iw1 == V_A) ? V_B : (S.iw1 == V_B ? V_C : V_A);
            Lane<double> Y = V(V_Y), F0 = V(V_F0), W1 = V(S.iw1), W2 = V(fin ? S.iw1 : S.iw2),
                         FJ = V(V_FX), WN = V(nw);
#pragma unroll 1
            for (int i = 0; i < L.nV; ++i)
                WN[i] = c0 * Y[i] + mu * W1[i] + nu * W2[i] + mt * FJ[i] + gt * F0[i];
        }
        const double acc = final_norm(S, fin, nw);
        if (sf) {
            if (fin) return rkc_final(S, acc);
            S.iw2 = S.iw1;
            S.iw1 = nw;
            S.in_v = nw;
            S.out_v = V_FX;
            if (S.j == S.s) S.phase = PH_FINAL;
            else S.j++;
            return -1;
        }
        if (S.phase == PH_SIGBASE) {
            sigma_start(S);
            return -1;
        }
        if (S.phase == PH_SIG) {
            if (!sigma_column(S)) return -1;
            if (!isfinite(S.sigma)) return KIN_CELL_NONFINITE;
            return rkc_begin_step(S);
        }
        if (S.phase == PH_POW) {
            if (!power_post(L.nV, V(V_Y), V(V_BASE), V(V_RS), V(V_X), V(V_FX), S.P)) return -1;
            S.sigma = 1.2 * S.P.sig;
            S.nsig++;
            S.since_sigma = 0;
            S.sigma_here = true;
            if (!isfinite(S.sigma)) return KIN_CELL_NONFINITE;
            return rkc_begin_step(S);
        }
        return -1;  // not reached: every RKC phase is handled above
    }

    // Step control after the final evaluation (Section 2.3): acc is the sum
    // of the squared weighted error components.
    __device__ int rkc_final(LaneState& S, double acc)
    {
        Lane<double> Y = V(V_Y), F0 = V(V_F0), WS = V(S.iw1), FX = V(V_FX);
        const double hh = S.hh;
        // x = ||Delta||^2: err <= 1 iff x <= 1, and the controller's powers
        // of err come from z = x^(-1/6) = err^(-1/3) (no square or cube root):
        // err^(1/3) = x z^5, err^(-2/3) = z^2.
        const double x = acc * S.invN;
        S.attempts++;
        if (x <= 1.0) {
            S.nacc++;
            double fac, c3 = 0.0;
            if (x == 0.0) {
                fac = 10.0;
            } else {
                const double z = rpow6_newton(x), z2 = z * z;
                c3 = x * (z2 * z2 * z);
                if (S.have_prev && !S.last_rejected && S.cprev > 0.0)
                    fac = 0.8 * hh * S.cprev * z2 * rcp_newton(S.hprev);
                else fac = 0.8 * z;
            }
            fac = fmin(10.0, fmax(0.1, fac));
#pragma unroll 1
            for (int i = 0; i < L.nV; ++i) {
                Y[i] = WS[i];
                F0[i] = FX[i];
            }
            if (S.last) {
                S.t = S.dt;
                return KIN_CELL_OK;
            }
            S.t += hh;  // err <= 1 implies f(w_s) is finite
            S.have_prev = true;
            S.hprev = hh;
            S.cprev = c3;
            S.last_rejected = false;
            S.sigma_here = false;
            S.since_sigma++;
            S.h = fac * hh;
        } else {
            S.nrej++;
            double fac = isfinite(x) ? 0.8 * rpow6_newton(x) : 0.1;
            if (fac < 0.1) fac = 0.1;
            S.last_rejected = true;
            S.h = fac * hh;
            if (S.h < 1e-20 * S.dt) return KIN_CELL_HMIN;
        }
        return rkc_begin_step(S);
    }

    // ------------------------------------------------------------ RKCK ---
    // Form stage point st (1..5): X = Y + hh sum_{l<st} b_{st,l} F_l.
    __device__ void rkck_stage_point(LaneState& S, int st)
    {
        Lane<double> Y = V(V_Y), X = V(V_X);
#pragma unroll 1
        for (int i = 0; i < L.nV; ++i) {
            double acc = 0.0;
            for (int l = 0; l < st; ++l) acc += CK_B[st][l] * V(ck_slot(l))[i];
            X[i] = Y[i] + S.hh * acc;
        }
        S.st = st;
        S.phase = PH_K;
        S.in_v = V_X;
        S.out_v = ck_slot(st);
    }

    __device__ int rkck_begin_attempt(LaneState& S)
    {
        if (S.attempts >= L.max_steps) return KIN_CELL_MAXSTEPS;
        double hh = S.h;
        S.last = false;
        if (hh >= S.dt - S.t) {
            hh = S.dt - S.t;
            S.last = true;
        }
        S.hh = hh;
        rkck_stage_point(S, 1);
        return -1;
    }

    __device__ int rkck_post(LaneState& S)
    {
        if (S.phase == PH_F0) {
            if (!finite_vec(V_F0)) return KIN_CELL_NONFINITE;
            return rkck_begin_attempt(S);
        }
        if (S.st < 5) {
            rkck_stage_point(S, S.st + 1);
            return -1;
        }
        // all six derivatives known: y5, error, errmax (Section 2.2)
        Lane<double> Y = V(V_Y), F0 = V(V_F0), X = V(V_X);
        const double hh = S.hh;
        double errmax = 0.0;
        bool blown = false;  // a NaN component makes the estimate non-finite (a rejection)
#pragma unroll 1
        for (int i = 0; i < L.nV; ++i) {
            double s5 = 0.0, e = 0.0;
            for (int l = 0; l < 6; ++l) {
                const double f = V(ck_slot(l))[i];
                s5 += CK_C[l] * f;
                e += CK_E[l] * f;
            }
            X[i] = Y[i] + hh * s5;
            const double tol = S.rtol * (fabs(Y[i]) + fabs(hh * F0[i])) + S.atol;
            const double r = fabs(hh * e) * rcp_newton(tol);
            blown |= isnan(r);
            if (r > errmax) errmax = r;
        }
        if (blown) errmax = __longlong_as_double(0x7ff8000000000000ll);
        S.attempts++;
        if (errmax <= 1.0) {
            S.nacc++;
#pragma unroll 1
            for (int i = 0; i < L.nV; ++i) Y[i] = X[i];
            if (S.last) {
                S.t = S.dt;
                return KIN_CELL_OK;
            }
            S.t += hh;
            const double hn = errmax == 0.0 ? 5.0 * hh : 0.9 * hh * rpow5_newton(errmax);
            S.h = fmin(hn, 5.0 * hh);
            S.phase = PH_F0;
            S.in_v = V_Y;
            S.out_v = V_F0;
            return -1;
        }
        S.nrej++;
        const double hn = isfinite(errmax) ? 0.9 * hh * rpow4_newton(errmax) : 0.1 * hh;
        S.h = fmax(hn, 0.1 * hh);
        if (S.h < 1e-20 * S.dt) return KIN_CELL_HMIN;
        return rkck_begin_attempt(S);
    }

    __device__ bool finite_vec(int v) const
    {
        Lane<double> a = V(v);
        bool ok = true;
#pragma unroll 1
        for (int i = 0; i < L.nV; ++i) ok &= isfinite(a[i]);
        return ok;
    }

    // --------------------------------------------------------- main loop --
    __device__ void run()
    {
        LaneState S;
        if (!load_next(S)) return;
        for (;;) {
            const bool sig = METHOD == KIN_RKC && S.phase >= PH_SIGBASE && S.phase <= PH_POW;
            if constexpr (EN) {
                if (!sig)
                    F::template eval_energy<R>(M, S.p, W.C, W.OM, V(S.in_v), V(S.out_v));
                else if constexpr (sizeof(R) == 4)
                    F::template eval_energy<double>(M, S.p, W.C64, W.OM64, V(S.in_v), V(S.out_v));
                else
                    F::template eval_energy<double>(M, S.p, W.C, W.OM, V(S.in_v), V(S.out_v));
            } else if (sizeof(R) == 4 && sig) {
                F::template eval<double, R>(M, S.Ctot, S.invCtot, K, KR, W.C64, W.OM64, V(S.in_v),
                                            V(S.out_v));
            } else {
                F::template eval<R, R>(M, S.Ctot, S.invCtot, K, KR, W.C, W.OM, V(S.in_v), V(S.out_v));
            }
            S.nfe++;
            S.nfs += sig;
            const int code = METHOD == KIN_RKC ? rkc_post(S) : rkck_post(S);
            if (code >= 0) {
                store(S, code);
                if (!load_next(S)) return;
            }
        }
    }
};

// OCC selects the register budget: 0 = at most 128 registers (16 resident
// warps per SM), 1 = at most 85 (24 resident warps per SM; the rarely used
// state spills to L1-backed local memory).
template <int METHOD, typename R, int STG, int OCC, bool EN, typename F = TableF>
__global__ void __launch_bounds__(128, OCC ? 6 : 4) integrate_kernel(const __grid_constant__ Launch L)
{
    const int64_t slot = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (slot >= L.nslots) return;
    Integrator<METHOD, R, STG, EN, F> I(L, slot);
    I.run();
}

#ifndef __CUDACC_RTC__

// ------------------------------------------------------- launch templates --
template <int METHOD, typename R, int STG, int OCC, bool EN>
inline cudaError_t launch_all(Launch& L, int blocks, int threads, cudaStream_t st)
{
    const size_t sm = smem_bytes(L.M, L.precision, threads, STG);
    if (STG > 0) {
        cudaError_t e = cudaFuncSetAttribute(init_kernel<METHOD, R, STG, EN>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(integrate_kernel<METHOD, R, STG, OCC, EN>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    init_kernel<METHOD, R, STG, EN><<<blocks, threads, sm, st>>>(L);
    if (METHOD == KIN_RKC) {
        const cudaError_t e = launch_sort(L, st);
        if (e != cudaSuccess) return e;
    }
    integrate_kernel<METHOD, R, STG, OCC, EN><<<blocks, threads, sm, st>>>(L);
    return cudaGetLastError();
}

template <int METHOD, typename R, int OCC>
inline cudaError_t launch_staged(Launch& L, int stg, int blocks, int threads, cudaStream_t st)
{
    if (stg == 2) return launch_all<METHOD, R, 2, OCC, false>(L, blocks, threads, st);
    if (stg == 1) return launch_all<METHOD, R, 1, OCC, false>(L, blocks, threads, st);
    return launch_all<METHOD, R, 0, OCC, false>(L, blocks, threads, st);
}

template <int METHOD, typename R>
inline cudaError_t launch_occ(Launch& L, int stg, int occ, int blocks, int threads, cudaStream_t st)
{
    return occ ? launch_staged<METHOD, R, 1>(L, stg, blocks, threads, st)
               : launch_staged<METHOD, R, 0>(L, stg, blocks, threads, st);
}

template <int METHOD, typename R, int STG, int OCC, bool EN = false>
inline cudaError_t occ_one(int threads, size_t sm, int* bps)
{
    if (STG > 0) {
        cudaError_t e = cudaFuncSetAttribute(integrate_kernel<METHOD, R, STG, OCC, EN>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, integrate_kernel<METHOD, R, STG, OCC, EN>,
                                                         threads, sm);
}

template <int METHOD, typename R, int OCC>
inline cudaError_t occ_staged(int stg, int threads, size_t sm, int* bps)
{
    if (stg == 2) return occ_one<METHOD, R, 2, OCC>(threads, sm, bps);
    if (stg == 1) return occ_one<METHOD, R, 1, OCC>(threads, sm, bps);
    return occ_one<METHOD, R, 0, OCC>(threads, sm, bps);
}

template <int METHOD, typename R>
inline cudaError_t occ_sel(int stg, int occ, int threads, size_t sm, int* bps)
{
    return occ ? occ_staged<METHOD, R, 1>(stg, threads, sm, bps)
               : occ_staged<METHOD, R, 0>(stg, threads, sm, bps);
}

// The energy-equation variants (staging level 0: their rate constants are
// formed inside f, so there is no per-lane copy to stage).
template <int METHOD, typename R>
inline cudaError_t launch_energy(Launch& L, int occ, int blocks, int threads, cudaStream_t st)
{
    return occ ? launch_all<METHOD, R, 0, 1, true>(L, blocks, threads, st)
               : launch_all<METHOD, R, 0, 0, true>(L, blocks, threads, st);
}

template <int METHOD, typename R>
inline cudaError_t occ_energy(int occ, int threads, size_t sm, int* bps)
{
    return occ ? occ_one<METHOD, R, 0, 1, true>(threads, sm, bps)
               : occ_one<METHOD, R, 0, 0, true>(threads, sm, bps);
}

#endif  // __CUDACC_RTC__

}  // namespace kin
