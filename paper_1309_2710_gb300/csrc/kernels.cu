// kernels.cu -- sm_103a kernels of the batched kinetics integrator.
//
// Design (one GB300, FP64-pipe bound):
//  * One lane integrates one cell (the cell's whole sub-stepping loop), as in
//    the paper's thread-per-ODE design (Section 3), but each loop iteration of
//    a lane performs exactly ONE evaluation of f. The method's control flow
//    (RKCK stages, RKC stages, finite-difference Jacobian columns, the initial
//    step probe, accept/reject) is a per-lane state machine around that single
//    call. Lanes of a warp in different phases or on cells with different
//    stage counts still execute the expensive part -- f -- together, so warp
//    divergence costs only the cheap bookkeeping, not whole f evaluations.
//  * The grid is persistent: lanes pull cells from a global atomic queue
//    (warp-aggregated), and a lane that finishes its cell immediately takes the
//    next one. Uneven cells (different step and stage counts) and uneven
//    instances therefore balance at lane granularity.
//  * Per-lane arrays (state vectors, rate constants, concentrations, rates of
//    progress) are element-major in the workspace: coalesced for a warp.
//  * f (Section 2.1): concentrations from the ideal gas law, Omega_j from the
//    hoisted rate constants (T is fixed over the flow step), third-body and
//    Lindemann falloff factors, and the stoichiometric sum as a gather over a
//    species-major CSR of the net coefficients (no scattered read-modify-
//    write). Template parameter R is the rate arithmetic type: double, or
//    float for the mixed-precision path (state and control stay double).
//  * No tensor cores: the stoichiometric contraction is sparse (about four
//    nonzeros per reaction).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "kin_dev.cuh"

namespace kin {

// ---------------------------------------------------------------- helpers --
template <typename T>
struct Lane {
    T* p;
    int64_t s;  // stride between elements (= lanes in the grid)
    __device__ __forceinline__ T& operator[](int i) const { return p[(int64_t)i * s]; }
};

template <typename R>
struct Tab;
template <>
struct Tab<double> {
    __device__ static const double* invW(const MechDev& M) { return M.invW; }
    __device__ static const double* eff(const MechDev& M) { return M.eff; }
    __device__ static const double* nu(const MechDev& M) { return M.csr_nu; }
    __device__ static double ex(double a) { return exp(a); }
};
template <>
struct Tab<float> {
    __device__ static const float* invW(const MechDev& M) { return M.invW32; }
    __device__ static const float* eff(const MechDev& M) { return M.eff32; }
    __device__ static const float* nu(const MechDev& M) { return M.csr_nu32; }
    __device__ static float ex(double a) { return expf((float)a); }
};

// Rate constants of one cell (Eq. (E:rxn-const)); T is fixed for the call.
// K_j = exp(ln A_j + beta_j ln T - (Ea_j/R)/T); for falloff reactions KR_j =
// k_0/k_inf. The exponent is formed in double; the exp runs in R.
template <typename R>
__device__ void rate_constants(const MechDev& M, double T, Lane<R> K, Lane<R> KR)
{
    const double lnT = log(T), invT = 1.0 / T;
    for (int j = 0; j < M.nR; ++j) {
        double a = M.lnA[j] + M.beta[j] * lnT - M.EaR[j] * invT;
        K[j] = Tab<R>::ex(a);
        if (M.rxn[j].type == KIN_RXN_FALLOFF) {
            double a0 = M.lnA0[j] + M.beta0[j] * lnT - M.Ea0R[j] * invT;
            KR[j] = Tab<R>::ex(a0 - a);
        }
    }
}

// f(x) -> out (Eqs. (E:mass), (E:spec-rate), (E:rxn-rate)). Ctot = p/(R T)
// in mol/cm^3. C and OM are lane scratch of nS and nR entries.
template <typename R>
__device__ void feval(const MechDev& M, double Ctot, Lane<R> K, Lane<R> KR, Lane<R> C,
                      Lane<R> OM, Lane<double> x, Lane<double> out)
{
    const int nS = M.nS, nR = M.nR;
    const R* __restrict__ invW = Tab<R>::invW(M);
    // mixture: S = sum Y/W = 1/Wbar, rho = Ctot Wbar, C_k = rho Y_k / W_k
    R S = R(0);
    for (int i = 0; i < nS; ++i) {
        R m = (R)x[i] * invW[i];
        C[i] = m;
        S += m;
    }
    const R rho = (R)Ctot / S;
    for (int i = 0; i < nS; ++i) C[i] = C[i] * rho;
    // rates of progress
    const R* __restrict__ eff = Tab<R>::eff(M);
    for (int j = 0; j < nR; ++j) {
        const Rxn r = M.rxn[j];
        R q = K[j];
        if (r.r0 >= 0) q *= C[r.r0];
        if (r.r1 >= 0) q *= C[r.r1];
        if (r.type != KIN_RXN_PLAIN) {
            const R* a = eff + (int64_t)r.row * nS;
            R Mc = R(0);
            for (int i = 0; i < nS; ++i) Mc += a[i] * C[i];
            if (r.type == KIN_RXN_THIRD_BODY) {
                q *= Mc;
            } else {
                R Pr = KR[j] * Mc;
                q *= Pr / (R(1) + Pr);
            }
        }
        OM[j] = q;
    }
    // omega_i = sum_j nu_ij Omega_j (gather), dY_i/dt = W_i omega_i / rho
    const R* __restrict__ nu = Tab<R>::nu(M);
    const double invrho = (double)S / Ctot;
    for (int i = 0; i < nS; ++i) {
        R w = R(0);
        const int e1 = M.csr_ptr[i + 1];
        for (int e = M.csr_ptr[i]; e < e1; ++e) w += nu[e] * OM[M.csr_rxn[e]];
        out[i] = (double)w * M.W[i] * invrho;
    }
}

// ------------------------------------------------------------ work queue --
// Warp-aggregated pop of the next global cell index for every active lane
// that calls it.
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

__device__ __forceinline__ int find_inst(const Launch& L, long long g)
{
    int lo = 0, hi = L.n_inst - 1;
    while (lo < hi) {  // largest i with start[i] <= g
        int mid = (lo + hi + 1) >> 1;
        if (L.start[mid] <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ------------------------------------------------------------ integrator --
enum Phase : int {
    PH_F0 = 0,   // f at the current accepted state -> F0
    PH_SIG,      // f at Y + eps_k e_k (Gershgorin column k) -> FX
    PH_PROBE,    // RKC initial step probe f(Y + h0 F0) -> FX
    PH_STAGE,    // RKC: f(w_{j-1}) -> FJ, then w_j
    PH_FINAL,    // RKC: f(w_s) -> FX, error estimate and control
    PH_K,        // RKCK: f at stage point -> F[st]
};

// Vector slots of the lane's working set.
enum Vec : int { V_Y = 0, V_F0, V_A, V_B, V_C, V_X, V_FX, V_RS };
// RKCK reuses slots: F[1..5] = V_A, V_B, V_C, V_FX, V_RS; the stage point is V_X.

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
    const int map[6] = {V_F0, V_A, V_B, V_C, V_FX, V_RS};
    return map[st];
}

struct LaneState {
    long long cell;  // local index within the instance
    int inst;
    int phase, st, j, s, col;
    int attempts, nacc, nrej, nsig, nfe;
    int since_sigma;
    bool initial, last, last_rejected, have_prev, sigma_here;
    int iw1, iw2;  // RKC: slots of w_{j-1}, w_{j-2}
    double t, dt, h, hh, h0, hprev, errprev, sigma, eps, rtol, atol, Ctot;
    int in_v, out_v;  // vectors read and written by the next f evaluation
};

template <int METHOD, typename R>
struct Integrator {
    const Launch& L;
    const MechDev& M;
    int64_t slot;
    Lane<R> K, KR, C, OM;
    double* vbase;

    __device__ Integrator(const Launch& l, int64_t sl) : L(l), M(l.M), slot(sl)
    {
        R* rb = reinterpret_cast<R*>(L.rarr) + sl;
        const int64_t s = L.nslots;
        K = Lane<R>{rb, s};
        KR = Lane<R>{rb + (int64_t)M.nR * s, s};
        C = Lane<R>{rb + (int64_t)2 * M.nR * s, s};
        OM = Lane<R>{rb + (int64_t)(2 * M.nR + M.nS) * s, s};
        vbase = L.vec + sl;
    }
    __device__ __forceinline__ Lane<double> V(int v) const
    {
        return Lane<double>{vbase + (int64_t)v * M.nS * L.nslots, L.nslots};
    }

    // ---------------------------------------------------------- cell I/O --
    __device__ bool load_next(LaneState& S)
    {
        const long long g = pop_cell(L.queue);
        if (g >= L.total) return false;
        const int i = find_inst(L, g);
        const InstDev& I = L.inst[i];
        S.inst = i;
        S.cell = g - L.start[i];
        const double T = I.T[S.cell], p = I.p[S.cell];
        Lane<double> Y = V(V_Y);
        for (int k = 0; k < M.nS; ++k) Y[k] = I.Y[(int64_t)k * I.ldY + S.cell];
        rate_constants<R>(M, T, K, KR);
        S.Ctot = p * 1e-6 / (R_GAS * T);
        S.dt = I.dt;
        S.rtol = I.rtol;
        S.atol = I.atol;
        S.t = 0.0;
        S.h = I.dt;
        S.attempts = S.nacc = S.nrej = S.nsig = S.nfe = 0;
        S.since_sigma = 0;
        S.initial = true;
        S.last = false;
        S.last_rejected = false;
        S.have_prev = false;
        S.sigma_here = false;
        S.hprev = S.errprev = S.sigma = 0.0;
        S.phase = PH_F0;
        S.in_v = V_Y;
        S.out_v = V_F0;
        return true;
    }

    __device__ void store(const LaneState& S, int code)
    {
        const InstDev& I = L.inst[S.inst];
        Lane<double> Y = V(V_Y);
        for (int k = 0; k < M.nS; ++k) I.Y[(int64_t)k * I.ldY + S.cell] = Y[k];
        if (I.status) I.status[S.cell] = (uint8_t)code;
        if (I.stats) {
            int32_t* st = I.stats + 4 * S.cell;
            st[0] = S.nfe;
            st[1] = S.nacc;
            st[2] = S.nrej;
            st[3] = S.nsig;
        }
    }

    // ----------------------------------------------------- shared pieces --
    __device__ bool finite_vec(int v) const
    {
        Lane<double> a = V(v);
        bool ok = true;
        for (int i = 0; i < M.nS; ++i) ok &= isfinite(a[i]);
        return ok;
    }

    // Weighted RMS norm, Eq. (E:rmsE), of d with T_i = atol + rtol max(|a|,|b|).
    __device__ double rms(const LaneState& S, Lane<double> d, Lane<double> a, Lane<double> b) const
    {
        double acc = 0.0;
        for (int i = 0; i < M.nS; ++i) {
            double sc = S.atol + S.rtol * fmax(fabs(a[i]), fabs(b[i]));
            double r = d[i] / sc;
            acc += r * r;
        }
        return sqrt(acc / M.nS);
    }

    // Start a Gershgorin estimate: X = Y + eps_0 e_0, RS = 0.
    __device__ void sigma_begin(LaneState& S)
    {
        Lane<double> Y = V(V_Y), X = V(V_X), RS = V(V_RS);
        for (int i = 0; i < M.nS; ++i) {
            X[i] = Y[i];
            RS[i] = 0.0;
        }
        S.col = 0;
        S.eps = sqrt_u() * fmax(fabs(Y[0]), S.atol);
        X[0] = Y[0] + S.eps;
        S.phase = PH_SIG;
        S.in_v = V_X;
        S.out_v = V_FX;
    }
    __device__ static double sqrt_u()
    {
        // sqrt of the unit roundoff of the rate arithmetic type
        return sizeof(R) == 8 ? 1.4901161193847656e-08 : 3.4526698300124393e-04;
    }

    // Post-processing of one Gershgorin column. Returns true when sigma is done.
    __device__ bool sigma_column(LaneState& S)
    {
        Lane<double> Y = V(V_Y), X = V(V_X), RS = V(V_RS), FX = V(V_FX), F0 = V(V_F0);
        const double e = S.eps;
        for (int i = 0; i < M.nS; ++i) RS[i] += fabs((FX[i] - F0[i]) / e);
        X[S.col] = Y[S.col];
        if (++S.col < M.nS) {
            S.eps = sqrt_u() * fmax(fabs(Y[S.col]), S.atol);
            X[S.col] = Y[S.col] + S.eps;
            return false;
        }
        double sg = 0.0;
        for (int i = 0; i < M.nS; ++i) sg = fmax(sg, RS[i]);
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

    // Choose the next attempt (or a spectral-radius refresh) after an
    // accepted/rejected step or the initial step. Returns a finish code >= 0
    // if the cell must stop, else -1.
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
        double sr = floor(1.0 + sqrt(1.0 + 1.54 * hh * S.sigma));
        int s;
        if (sr < 2.0) {
            s = 2;
        } else if (sr > (double)SMAX) {
            s = SMAX;
            hh = ((SMAX - 1.0) * (SMAX - 1.0) - 1.0) / (1.54 * S.sigma);
            S.last = false;
        } else {
            s = (int)sr;
        }
        S.hh = hh;
        S.s = s;
        // w_1 = y + mu~_1 h f_0 into slot A; w_0 = y stays in V_Y
        const double m1 = coef(s, 1)[2] * hh;
        Lane<double> Y = V(V_Y), F0 = V(V_F0), A = V(V_A);
        for (int i = 0; i < M.nS; ++i) A[i] = Y[i] + m1 * F0[i];
        S.iw1 = V_A;
        S.iw2 = V_Y;
        S.j = 2;
        S.phase = PH_STAGE;
        S.in_v = V_A;
        S.out_v = V_FX;
        return -1;
    }

    __device__ int rkc_post(LaneState& S)
    {
        switch (S.phase) {
        case PH_F0: {
            if (!finite_vec(V_F0)) return KIN_CELL_NONFINITE;
            sigma_begin(S);
            return -1;
        }
        case PH_SIG: {
            if (!sigma_column(S)) return -1;
            if (!isfinite(S.sigma)) return KIN_CELL_NONFINITE;
            if (!S.initial) return rkc_begin_step(S);
            // initial step: h0 = 1/sigma, probe f(y + h0 f0)
            double h0 = S.sigma > 0.0 ? 1.0 / S.sigma : S.dt;
            if (h0 > S.dt) h0 = S.dt;
            S.h0 = h0;
            Lane<double> Y = V(V_Y), F0 = V(V_F0), X = V(V_X);
            for (int i = 0; i < M.nS; ++i) X[i] = Y[i] + h0 * F0[i];
            S.phase = PH_PROBE;
            S.in_v = V_X;
            S.out_v = V_FX;
            return -1;
        }
        case PH_PROBE: {
            Lane<double> Y = V(V_Y), F0 = V(V_F0), FX = V(V_FX), D = V(V_X);
            for (int i = 0; i < M.nS; ++i) D[i] = S.h0 * (FX[i] - F0[i]);
            const double e0 = rms(S, D, Y, Y);
            double h;
            if (!isfinite(e0)) h = 0.1 * S.h0;
            else h = e0 > 0.0 ? 0.1 * S.h0 / sqrt(e0) : S.dt;
            if (h > S.dt) h = S.dt;
            if (h < 1e-20 * S.dt) return KIN_CELL_HMIN;
            S.h = h;
            S.initial = false;
            return rkc_begin_step(S);
        }
        case PH_STAGE: {
            // FX = f(w_{j-1}); w_j = (1-mu-nu) y + mu w_{j-1} + nu w_{j-2}
            //                       + mu~ h f_{j-1} + gamma~ h f_0
            const double* c = coef(S.s, S.j);
            const double mu = c[0], nu = c[1], mt = c[2] * S.hh, gt = c[3] * S.hh, c0 = c[4];
            const int nw = (S.iw1 == V_A) ? V_B : (S.iw1 == V_B ? V_C : V_A);
            Lane<double> Y = V(V_Y), F0 = V(V_F0), W1 = V(S.iw1), W2 = V(S.iw2), FJ = V(V_FX),
                         WN = V(nw);
            for (int i = 0; i < M.nS; ++i)
                WN[i] = c0 * Y[i] + mu * W1[i] + nu * W2[i] + mt * FJ[i] + gt * F0[i];
            S.iw2 = S.iw1;
            S.iw1 = nw;
            S.in_v = nw;
            S.out_v = V_FX;
            if (S.j == S.s) S.phase = PH_FINAL;
            else S.j++;
            return -1;
        }
        case PH_FINAL: {
            // error estimate (Section 2.3) and step control
            Lane<double> Y = V(V_Y), F0 = V(V_F0), WS = V(S.iw1), FX = V(V_FX);
            double acc = 0.0;
            const double hh = S.hh;
            for (int i = 0; i < M.nS; ++i) {
                double d = 0.8 * (Y[i] - WS[i]) + 0.4 * hh * (F0[i] + FX[i]);
                double sc = S.atol + S.rtol * fmax(fabs(Y[i]), fabs(WS[i]));
                double r = d / sc;
                acc += r * r;
            }
            const double err = sqrt(acc / M.nS);
            S.attempts++;
            if (err <= 1.0) {
                S.nacc++;
                double fac;
                if (err == 0.0) fac = 10.0;
                else if (S.have_prev && !S.last_rejected && S.errprev > 0.0)
                    fac = 0.8 * (hh / S.hprev) * cbrt(S.errprev) / pow(err, 2.0 / 3.0);
                else fac = 0.8 / cbrt(err);
                fac = fmin(10.0, fmax(0.1, fac));
                for (int i = 0; i < M.nS; ++i) {
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
                S.errprev = err;
                S.last_rejected = false;
                S.sigma_here = false;
                S.since_sigma++;
                S.h = fac * hh;
            } else {
                S.nrej++;
                double fac = isfinite(err) ? 0.8 / cbrt(err) : 0.1;
                if (fac < 0.1) fac = 0.1;
                S.last_rejected = true;
                S.h = fac * hh;
                if (S.h < 1e-20 * S.dt) return KIN_CELL_HMIN;
            }
            return rkc_begin_step(S);
        }
        default:
            return KIN_CELL_NONFINITE;
        }
    }

    // ------------------------------------------------------------ RKCK ---
    // Form stage point st (1..5): X = Y + hh sum_{l<st} b_{st,l} F_l.
    __device__ void rkck_stage_point(LaneState& S, int st)
    {
        Lane<double> Y = V(V_Y), X = V(V_X);
        for (int i = 0; i < M.nS; ++i) {
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
        // PH_K
        if (S.st < 5) {
            rkck_stage_point(S, S.st + 1);
            return -1;
        }
        // all six derivatives known: y5, error, errmax (Section 2.2)
        Lane<double> Y = V(V_Y), F0 = V(V_F0), X = V(V_X);
        const double hh = S.hh;
        double errmax = 0.0;
        for (int i = 0; i < M.nS; ++i) {
            double s5 = 0.0, e = 0.0;
            for (int l = 0; l < 6; ++l) {
                const double f = V(ck_slot(l))[i];
                s5 += CK_C[l] * f;
                e += CK_E[l] * f;
            }
            X[i] = Y[i] + hh * s5;
            const double tol = S.rtol * (fabs(Y[i]) + fabs(hh * F0[i])) + S.atol;
            const double r = fabs(hh * e) / tol;
            if (!(r <= errmax)) errmax = r;
        }
        S.attempts++;
        if (errmax <= 1.0) {
            S.nacc++;
            for (int i = 0; i < M.nS; ++i) Y[i] = X[i];
            if (S.last) {
                S.t = S.dt;
                return KIN_CELL_OK;
            }
            S.t += hh;
            double hn = errmax == 0.0 ? 5.0 * hh : 0.9 * hh * pow(errmax, -0.2);
            S.h = fmin(hn, 5.0 * hh);
            S.phase = PH_F0;
            S.in_v = V_Y;
            S.out_v = V_F0;
            return -1;
        }
        S.nrej++;
        double hn = isfinite(errmax) ? 0.9 * hh * pow(errmax, -0.25) : 0.1 * hh;
        S.h = fmax(hn, 0.1 * hh);
        if (S.h < 1e-20 * S.dt) return KIN_CELL_HMIN;
        return rkck_begin_attempt(S);
    }

    // --------------------------------------------------------- main loop --
    __device__ void run()
    {
        LaneState S;
        if (!load_next(S)) return;
        for (;;) {
            feval<R>(M, S.Ctot, K, KR, C, OM, V(S.in_v), V(S.out_v));
            S.nfe++;
            const int code = METHOD == KIN_RKC ? rkc_post(S) : rkck_post(S);
            if (code >= 0) {
                store(S, code);
                if (!load_next(S)) return;
            }
        }
    }
};

template <int METHOD, typename R>
__global__ void __launch_bounds__(128) integrate_kernel(const __grid_constant__ Launch L)
{
    const int64_t slot = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (slot >= L.nslots) return;
    Integrator<METHOD, R> I(L, slot);
    I.run();
}

// ------------------------------------------------------------- f alone ---
template <typename R>
__global__ void rates_kernel(MechDev M, int64_t cells, const double* __restrict__ T,
                             const double* __restrict__ p, const double* Y, int64_t ldY,
                             double* dYdt, void* rarr, int64_t nslots)
{
    const int64_t slot = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (slot >= nslots) return;
    R* rb = reinterpret_cast<R*>(rarr) + slot;
    Lane<R> K{rb, nslots}, KR{rb + (int64_t)M.nR * nslots, nslots},
        C{rb + (int64_t)2 * M.nR * nslots, nslots},
        OM{rb + (int64_t)(2 * M.nR + M.nS) * nslots, nslots};
    for (int64_t c = slot; c < cells; c += nslots) {
        rate_constants<R>(M, T[c], K, KR);
        const double Ctot = p[c] * 1e-6 / (R_GAS * T[c]);
        feval<R>(M, Ctot, K, KR, C, OM, Lane<double>{const_cast<double*>(Y) + c, ldY},
                 Lane<double>{dYdt + c, ldY});
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
    // first pass: T', T'' at j = s for w1
    double t0 = 1.0, t1 = w0, d0 = 0.0, d1 = 1.0, e0 = 0.0, e1 = 0.0;
    for (int j = 2; j <= s; ++j) {
        double t2 = 2.0 * w0 * t1 - t0;
        double d2 = 2.0 * t1 + 2.0 * w0 * d1 - d0;
        double e2 = 4.0 * d1 + 2.0 * w0 * e1 - e0;
        t0 = t1; t1 = t2; d0 = d1; d1 = d2; e0 = e1; e1 = e2;
    }
    const double w1 = d1 / e1;
    // second pass: coefficients
    t0 = 1.0; t1 = w0; d0 = 0.0; d1 = 1.0; e0 = 0.0; e1 = 0.0;
    const double b2 = 4.0 / (16.0 * w0 * w0);  // T_2''/T_2'^2 = 4 / (4 w0)^2
    double bjm2 = b2, bjm1 = b2;  // b_0, b_1
    double ajm1 = 1.0 - b2 * w0;  // a_1 = 1 - b_1 T_1(w0)
    double* row1 = tab + ((int64_t)s * RKC_TAB_S + 1) * RKC_TAB_W;
    row1[0] = row1[1] = row1[3] = row1[4] = 0.0;
    row1[2] = b2 * w1;
    for (int j = 2; j <= s; ++j) {
        double t2 = 2.0 * w0 * t1 - t0;
        double d2 = 2.0 * t1 + 2.0 * w0 * d1 - d0;
        double e2 = 4.0 * d1 + 2.0 * w0 * e1 - e0;
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
int64_t scratch_elems_vec(int nS) { return (int64_t)NVEC * nS; }

int64_t scratch_bytes_rate(int nS, int nR, int precision)
{
    const int64_t n = (int64_t)3 * nR + nS;
    return n * (precision == KIN_MIXED ? 4 : 8);
}

template <int METHOD, typename R>
static cudaError_t launch_one(const Launch& L, int blocks, int threads, cudaStream_t st)
{
    integrate_kernel<METHOD, R><<<blocks, threads, 0, st>>>(L);
    return cudaGetLastError();
}

cudaError_t launch_integrate(const Launch& L, int blocks, int threads, cudaStream_t st)
{
    if (L.method == KIN_RKCK)
        return L.precision == KIN_MIXED ? launch_one<KIN_RKCK, float>(L, blocks, threads, st)
                                        : launch_one<KIN_RKCK, double>(L, blocks, threads, st);
    return L.precision == KIN_MIXED ? launch_one<KIN_RKC, float>(L, blocks, threads, st)
                                    : launch_one<KIN_RKC, double>(L, blocks, threads, st);
}

cudaError_t integrate_occupancy(int method, int precision, int threads, int* bps)
{
    if (method == KIN_RKCK)
        return precision == KIN_MIXED
                   ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, integrate_kernel<KIN_RKCK, float>, threads, 0)
                   : cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, integrate_kernel<KIN_RKCK, double>, threads, 0);
    return precision == KIN_MIXED
               ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, integrate_kernel<KIN_RKC, float>, threads, 0)
               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, integrate_kernel<KIN_RKC, double>, threads, 0);
}

cudaError_t launch_rates(const MechDev& M, int64_t cells, const double* T, const double* p,
                         const double* Y, int64_t ldY, double* dYdt, int precision, void* rarr,
                         int64_t nslots, int blocks, int threads, cudaStream_t st)
{
    if (precision == KIN_MIXED)
        rates_kernel<float><<<blocks, threads, 0, st>>>(M, cells, T, p, Y, ldY, dYdt, rarr, nslots);
    else
        rates_kernel<double><<<blocks, threads, 0, st>>>(M, cells, T, p, Y, ldY, dYdt, rarr, nslots);
    return cudaGetLastError();
}

cudaError_t launch_rkc_table(double* tab, cudaStream_t st)
{
    rkc_table_kernel<<<(SMAX + 1 + 127) / 128, 128, 0, st>>>(tab);
    return cudaGetLastError();
}

}  // namespace kin
