/*
 * kin_oracle.c -- plain, slow FP64 reference of the batched kinetics integrator.
 *
 * TEST INFRASTRUCTURE. Only the tests, the smoke check and the CPU baseline leg
 * of the benchmark load this library. The product path never calls it, and it
 * shares no code, header, table or constant with the CUDA implementation.
 *
 * What it computes (Niemeyer & Sung, "Accelerating moderately stiff chemical
 * kinetics in reactive-flow simulations using GPUs"):
 *   f      species source terms, Section 2.1, Eqs. (E:mass), (E:spec-rate),
 *          (E:rxn-rate), (E:rxn-const), with third-body and Lindemann falloff
 *          terms in the Chemkin form the paper refers to.
 *   RKCK   Cash-Karp 5(4) with the error test and step rule of Section 2.2,
 *          Table 1 (T:rkck) and Eq. (E:hnew).
 *   RKC    second-order Runge-Kutta-Chebyshev of Section 2.3: stage recursion
 *          Eqs. (E:rkc0)-(E:rkcs), coefficients, error estimate, RMS norm
 *          Eq. (E:rmsE), step controller, initial step and stage count, with the
 *          spectral radius from a Gershgorin bound on a finite-difference
 *          Jacobian (the alternative named at the end of Section 2.3).
 *
 * Readings where the paper is silent, garbled or inconsistent:
 *   - Temperature is held fixed over the flow step (no energy equation), so
 *     N = n_S and every k_j is constant within one call.
 *   - Density and concentrations follow the ideal gas law:
 *       rho = p Wbar / (R T) * 1e-6  [g/cm^3],  C_k = rho Y_k / W_k [mol/cm^3].
 *   - Lindemann falloff: Omega = k_inf * Pr/(1+Pr) * prod C, Pr = k_0 [M]/k_inf,
 *     without an extra [M] factor. A third-body reaction multiplies by [M].
 *   - RKCK: first trial step = the flow step; Delta_0,i = rtol(|y_i| +
 *     |h f_i(y_n)|) + atol; errmax = max_i |Delta_i| / Delta_0,i; accept iff
 *     errmax <= 1; growth limited to 5x, shrink to 10x.
 *   - RKC: b_0 = b_1 = b_2 (makes c_1 = c_2 / T_2'(w0) hold);
 *     a_j = 1 - b_j T_j(w0); controller on accept after an accepted step
 *     fac = 0.8 (h_n/h_{n-1}) err_n^{1/3} / err_{n+1}^{2/3}, otherwise
 *     fac = 0.8 / err^{1/3}; fac clamped to [0.1, 10]; err == 0 gives 10.
 *   - Stage count s = max(2, floor(1 + sqrt(1 + 1.54 h sigma))); s <= 250,
 *     with h reduced to ((250-1)^2 - 1)/(1.54 sigma) when capped.
 *   - sigma is estimated before the first step, before the step following 25
 *     accepted steps since the last estimate, and after a rejection when the
 *     last estimate was made at an earlier point (re-estimating at the same
 *     point gives the same bound).
 *   - Spectral radius: the Gershgorin bound (below), or the nonlinear power
 *     method (power_sigma) that the paper used; both are re-estimated on the
 *     same schedule.
 *   - Gershgorin: sigma = max_i sum_k |J_ik| with
 *     J_ik = (f_i(y + eps_k e_k) - f_i(y)) / eps_k,
 *     eps_k = sqrt(2^-52) * max(|y_k|, atol).
 *   - Every step is clipped to the end of the flow step; hmin = 1e-20 * dt.
 *   - A non-finite error estimate (a trial step that blew up) is a rejection
 *     with the largest decrease (0.1); a non-finite initial-step estimate
 *     gives h = 0.1 h0.
 *
 * Energy equation (Eq. (E:energy)), used when a call asks for it and the
 * mechanism has thermochemistry (orc_mech_set_thermo):
 *   - the state is y = {Y_1..Y_nS, T} (the paper lists T first; the order of
 *     the components changes neither the RMS norm, nor the Gershgorin bound,
 *     nor the power method), N = nS + 1;
 *   - dT/dt = -(1 / (rho cp)) sum_i h_i omega_i W_i, with the mass-averaged
 *     cp = sum_i Y_i cp_i / W_i and the specific enthalpy h_i = H_i / W_i;
 *   - the thermochemistry of the synthetic mechanisms is one constant molar
 *     heat capacity cp_i [J/(mol K)] and formation enthalpy Hf_i [J/mol] at
 *     298.15 K per species: H_i(T) = Hf_i + cp_i (T - 298.15);
 *   - k_j, rho and the concentrations follow T at every evaluation of f.
 *
 * Per-cell status codes: 0 ok, 1 step limit reached, 2 step size below hmin,
 * 3 non-finite f at an accepted state (or at the initial state), or a
 * non-finite spectral-radius bound. On 1-3 the cell keeps its last accepted
 * state.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_R 8.314462618 /* J/(mol K) */

typedef struct {
    int nS, nR;
    double *W;                 /* [nS] g/mol */
    double *lnA, *beta, *Ea;   /* [nR] forward Arrhenius */
    double *lnA0, *beta0, *Ea0;/* [nR] low-pressure limit (falloff only) */
    int *reac, *prod;          /* [nR][2], -1 = empty slot */
    int *type;                 /* [nR] 0 plain, 1 third body, 2 falloff */
    int *row;                  /* [nR] efficiency row or -1 */
    double *eff;               /* [n_rows][nS] */
    double *cp, *Hf;           /* [nS] J/(mol K), J/mol at ORC_TREF; NULL without thermo */
} orc_mech;

#define ORC_TREF 298.15 /* K */

static void *xmalloc(size_t n) { void *p = malloc(n ? n : 1); return p; }

static int all_finite(int n, const double *v)
{
    int i;
    for (i = 0; i < n; i++)
        if (!isfinite(v[i])) return 0;
    return 1;
}

void *orc_mech_new(int nS, int nR, const double *W, const double *lnA,
                   const double *beta, const double *Ea, const int32_t *reac,
                   const int32_t *prod, const int8_t *type, const double *eff,
                   const double *lnA0, const double *beta0, const double *Ea0)
{
    orc_mech *m = (orc_mech *)xmalloc(sizeof(orc_mech));
    int j, rows = 0;
    m->nS = nS;
    m->nR = nR;
    m->W = (double *)xmalloc(sizeof(double) * nS);
    memcpy(m->W, W, sizeof(double) * nS);
    m->lnA = (double *)xmalloc(sizeof(double) * nR);
    m->beta = (double *)xmalloc(sizeof(double) * nR);
    m->Ea = (double *)xmalloc(sizeof(double) * nR);
    m->lnA0 = (double *)xmalloc(sizeof(double) * nR);
    m->beta0 = (double *)xmalloc(sizeof(double) * nR);
    m->Ea0 = (double *)xmalloc(sizeof(double) * nR);
    m->reac = (int *)xmalloc(sizeof(int) * 2 * nR);
    m->prod = (int *)xmalloc(sizeof(int) * 2 * nR);
    m->type = (int *)xmalloc(sizeof(int) * nR);
    m->row = (int *)xmalloc(sizeof(int) * nR);
    for (j = 0; j < nR; j++) {
        m->lnA[j] = lnA[j];
        m->beta[j] = beta[j];
        m->Ea[j] = Ea[j];
        m->lnA0[j] = lnA0 ? lnA0[j] : 0.0;
        m->beta0[j] = beta0 ? beta0[j] : 0.0;
        m->Ea0[j] = Ea0 ? Ea0[j] : 0.0;
        m->reac[2 * j] = reac[2 * j];
        m->reac[2 * j + 1] = reac[2 * j + 1];
        m->prod[2 * j] = prod[2 * j];
        m->prod[2 * j + 1] = prod[2 * j + 1];
        m->type[j] = type[j];
        m->row[j] = type[j] != 0 ? rows++ : -1;
    }
    m->eff = (double *)xmalloc(sizeof(double) * (size_t)rows * nS);
    if (rows) memcpy(m->eff, eff, sizeof(double) * (size_t)rows * nS);
    m->cp = NULL;
    m->Hf = NULL;
    return m;
}

/* Species thermochemistry for the energy equation: constant molar heat
 * capacities cp [J/(mol K)] and formation enthalpies Hf [J/mol] at 298.15 K. */
void orc_mech_set_thermo(void *mp, const double *cp, const double *Hf)
{
    orc_mech *m = (orc_mech *)mp;
    free(m->cp);
    free(m->Hf);
    m->cp = (double *)xmalloc(sizeof(double) * m->nS);
    m->Hf = (double *)xmalloc(sizeof(double) * m->nS);
    memcpy(m->cp, cp, sizeof(double) * m->nS);
    memcpy(m->Hf, Hf, sizeof(double) * m->nS);
}

void orc_mech_free(void *p)
{
    orc_mech *m = (orc_mech *)p;
    if (!m) return;
    free(m->W); free(m->lnA); free(m->beta); free(m->Ea);
    free(m->lnA0); free(m->beta0); free(m->Ea0);
    free(m->reac); free(m->prod); free(m->type); free(m->row); free(m->eff);
    free(m->cp); free(m->Hf);
    free(m);
}

/* Eq. (E:rxn-const): k = A T^beta exp(-E / (R T)), for the forward rate and,
 * for falloff reactions, the low-pressure limit. */
void orc_rate_constants(const void *mp, double T, double *k, double *k0)
{
    const orc_mech *m = (const orc_mech *)mp;
    int j;
    for (j = 0; j < m->nR; j++) {
        k[j] = exp(m->lnA[j]) * pow(T, m->beta[j]) * exp(-m->Ea[j] / (ORC_R * T));
        if (m->type[j] == 2)
            k0[j] = exp(m->lnA0[j]) * pow(T, m->beta0[j]) * exp(-m->Ea0[j] / (ORC_R * T));
        else
            k0[j] = 0.0;
    }
}

/* Molar production rates omega [mol/(cm^3 s)] (Eqs. (E:spec-rate),
 * (E:rxn-rate)) and the density rho [g/cm^3] at T, p, Y; k, k0 from
 * orc_rate_constants at the same T. C: nS doubles of scratch. */
static double production(const orc_mech *m, double T, double p, const double *k,
                         const double *k0, const double *Y, double *omega, double *C)
{
    int nS = m->nS, i, j, s;
    double sum = 0.0, Wbar, rho;
    for (i = 0; i < nS; i++) sum += Y[i] / m->W[i];
    Wbar = 1.0 / sum;
    rho = p * Wbar / (ORC_R * T) * 1e-6;
    for (i = 0; i < nS; i++) C[i] = rho * Y[i] / m->W[i];
    for (i = 0; i < nS; i++) omega[i] = 0.0;
    for (j = 0; j < m->nR; j++) {
        double q = k[j];
        for (s = 0; s < 2; s++)
            if (m->reac[2 * j + s] >= 0) q *= C[m->reac[2 * j + s]];
        if (m->type[j] != 0) {
            const double *a = m->eff + (size_t)m->row[j] * nS;
            double M = 0.0;
            for (i = 0; i < nS; i++) M += a[i] * C[i];
            if (m->type[j] == 1) {
                q *= M;
            } else {
                double Pr = k0[j] * M / k[j];
                q *= Pr / (1.0 + Pr);
            }
        }
        /* omega_i = sum_j (nu''_ij - nu'_ij) Omega_j */
        for (s = 0; s < 2; s++) {
            if (m->prod[2 * j + s] >= 0) omega[m->prod[2 * j + s]] += q;
            if (m->reac[2 * j + s] >= 0) omega[m->reac[2 * j + s]] -= q;
        }
    }
    return rho;
}

/* f: dY/dt at fixed T and p, Eq. (E:mass). k, k0 from orc_rate_constants at
 * the same T. work: 2 nS doubles. */
static void rates(const orc_mech *m, double T, double p, const double *k,
                  const double *k0, const double *Y, double *dYdt, double *work)
{
    int i;
    double *C = work, *omega = work + m->nS;
    double rho = production(m, T, p, k, k0, Y, omega, C);
    for (i = 0; i < m->nS; i++) dYdt[i] = m->W[i] * omega[i] / rho;
}

/* f with the energy equation: y = {Y_1..Y_nS, T} -> dy/dt, Eqs. (E:mass) and
 * (E:energy). The rate constants, density and concentrations are those of the
 * state's own T. work: 2 nS + 2 nR doubles. */
static void rates_energy(const orc_mech *m, double p, const double *y, double *dydt,
                         double *work)
{
    int i, nS = m->nS;
    double *C = work, *omega = work + nS, *k = work + 2 * nS, *k0 = k + m->nR;
    double T = y[nS], rho, cpm = 0.0, hw = 0.0;
    orc_rate_constants(m, T, k, k0);
    rho = production(m, T, p, k, k0, y, omega, C);
    for (i = 0; i < nS; i++) {
        dydt[i] = m->W[i] * omega[i] / rho;
        cpm += y[i] * m->cp[i] / m->W[i];                     /* J/(g K) */
        hw += (m->Hf[i] + m->cp[i] * (T - ORC_TREF)) * omega[i]; /* h_i W_i omega_i, J/(cm^3 s) */
    }
    dydt[nS] = -hw / (rho * cpm);
}

/* Public f with the energy equation for tests: y = {Y, T} -> dy/dt. */
void orc_rates_energy(const void *mp, double p, const double *y, double *dydt)
{
    const orc_mech *m = (const orc_mech *)mp;
    double *work = (double *)xmalloc(sizeof(double) * (2 * m->nS + 2 * m->nR));
    rates_energy(m, p, y, dydt, work);
    free(work);
}

/* Public f for tests: computes k at T, then dY/dt. */
void orc_rates(const void *mp, double T, double p, const double *Y, double *dYdt)
{
    const orc_mech *m = (const orc_mech *)mp;
    double *k = (double *)xmalloc(sizeof(double) * 2 * m->nR);
    double *work = (double *)xmalloc(sizeof(double) * 2 * m->nS);
    orc_rate_constants(m, T, k, k + m->nR);
    rates(m, T, p, k, k + m->nR, Y, dYdt, work);
    free(k);
    free(work);
}

/* ---------------------------------------------------------------- RKCK --- */
/* Table 1 (T:rkck): a_i, b_ij, c_i, c*_i. */
static const double RK_A[6] = {0.0, 1.0 / 5.0, 3.0 / 10.0, 3.0 / 5.0, 1.0, 7.0 / 8.0};
static const double RK_B[6][5] = {
    {0, 0, 0, 0, 0},
    {1.0 / 5.0, 0, 0, 0, 0},
    {3.0 / 40.0, 9.0 / 40.0, 0, 0, 0},
    {3.0 / 10.0, -9.0 / 10.0, 6.0 / 5.0, 0, 0},
    {-11.0 / 54.0, 5.0 / 2.0, -70.0 / 27.0, 35.0 / 27.0, 0},
    {1631.0 / 55296.0, 175.0 / 512.0, 575.0 / 13824.0, 44275.0 / 110592.0, 253.0 / 4096.0}};
static const double RK_C[6] = {37.0 / 378.0, 0.0, 250.0 / 621.0, 125.0 / 594.0, 0.0, 512.0 / 1771.0};
static const double RK_CS[6] = {2825.0 / 27648.0, 0.0, 18575.0 / 48384.0, 13525.0 / 55296.0,
                                277.0 / 14336.0, 1.0 / 4.0};

void orc_rkck_table(double *a, double *b, double *c, double *cs)
{
    int i, j;
    for (i = 0; i < 6; i++) {
        a[i] = RK_A[i];
        c[i] = RK_C[i];
        cs[i] = RK_CS[i];
        for (j = 0; j < 5; j++) b[5 * i + j] = RK_B[i][j];
    }
}

/* The right-hand side of one cell: isothermal (T fixed, k precomputed) or,
 * with `energy`, the coupled species and energy equations. */
typedef struct {
    const orc_mech *m;
    double T, p;
    const double *k, *k0;
    double *work;              /* 2 nS + 2 nR doubles */
    int energy;
    long nfe;
} orc_f;

static void feval(orc_f *F, const double *y, double *out)
{
    if (F->energy)
        rates_energy(F->m, F->p, y, out, F->work);
    else
        rates(F->m, F->T, F->p, F->k, F->k0, y, out, F->work);
    F->nfe++;
}

/* One Cash-Karp step of size h from y with f0 = f(y): the formulas of
 * Section 2.2. Writes the fifth-order solution and err = y5 - y4.
 * kk: 6*nS doubles, x: nS doubles. */
static void rkck_step(orc_f *F, int n, const double *y, const double *f0, double h,
                      double *y5, double *err, double *kk, double *x)
{
    int i, l, st;
    for (i = 0; i < n; i++) kk[i] = h * f0[i];
    for (st = 1; st < 6; st++) {
        for (i = 0; i < n; i++) {
            double acc = y[i];
            for (l = 0; l < st; l++) acc += RK_B[st][l] * kk[l * n + i];
            x[i] = acc;
        }
        feval(F, x, kk + st * n);
        for (i = 0; i < n; i++) kk[st * n + i] *= h;
    }
    for (i = 0; i < n; i++) {
        double s5 = y[i], e = 0.0;
        for (l = 0; l < 6; l++) {
            s5 += RK_C[l] * kk[l * n + i];
            e += (RK_C[l] - RK_CS[l]) * kk[l * n + i];
        }
        y5[i] = s5;
        err[i] = e;
    }
}

/* Per-cell counters, and an optional per-attempt trace (step size tried,
 * error measure, stage count or 0 for RKCK, 1 if accepted, and the spectral
 * radius the RKC stage count was taken from, 0 for RKCK) used by tests. */
typedef struct {
    int nfe, nacc, nrej, nsig, nfs; /* nfs: f evaluations inside sigma estimates */
    int cap, len;
    double *tr_h, *tr_err, *tr_sig;
    int *tr_s, *tr_acc;
} orc_stats;

static void trace(orc_stats *st, double h, double err, int s, int acc, double sigma)
{
    if (st->len < st->cap) {
        st->tr_h[st->len] = h;
        st->tr_err[st->len] = err;
        st->tr_s[st->len] = s;
        st->tr_acc[st->len] = acc;
        if (st->tr_sig) st->tr_sig[st->len] = sigma;
    }
    st->len++;
}

static int rkck_cell(orc_f *F, int n, double *y, double dt, double rtol, double atol,
                     int max_steps, orc_stats *st)
{
    double *f0 = (double *)xmalloc(sizeof(double) * n * 10);
    double *y5 = f0 + n, *err = y5 + n, *x = err + n, *kk = x + n;
    double t = 0.0, h = dt, hmin = 1e-20 * dt;
    int i, attempts = 0, status = 0;
    feval(F, y, f0);
    if (!all_finite(n, f0)) { free(f0); return 3; }
    for (;;) {
        double hh = h, errmax = 0.0, hnew;
        int last = 0;
        if (attempts >= max_steps) { status = 1; break; }
        if (hh >= dt - t) { hh = dt - t; last = 1; }
        rkck_step(F, n, y, f0, hh, y5, err, kk, x);
        attempts++;
        for (i = 0; i < n; i++) {
            double tol = rtol * (fabs(y[i]) + fabs(hh * f0[i])) + atol;
            double r = fabs(err[i]) / tol;
            if (isnan(r)) { errmax = NAN; break; } /* a blown-up component: reject */
            if (r > errmax) errmax = r;
        }
        trace(st, hh, errmax, 0, errmax <= 1.0, 0.0);
        if (errmax <= 1.0) {
            st->nacc++;
            memcpy(y, y5, sizeof(double) * n);
            t = last ? dt : t + hh;
            if (last) break;
            hnew = errmax == 0.0 ? 5.0 * hh : 0.9 * hh * pow(errmax, -0.2);
            if (hnew > 5.0 * hh) hnew = 5.0 * hh;
            feval(F, y, f0);
            if (!all_finite(n, f0)) { status = 3; break; }
        } else {
            /* a non-finite estimate (the trial step blew up) is a rejection
             * with the largest decrease */
            st->nrej++;
            hnew = isfinite(errmax) ? 0.9 * hh * pow(errmax, -0.25) : 0.1 * hh;
            if (hnew < 0.1 * hh) hnew = 0.1 * hh;
            if (hnew < hmin) { status = 2; break; }
        }
        h = hnew;
    }
    free(f0);
    return status;
}

/* ----------------------------------------------------------------- RKC --- */
#define ORC_KAPPA (2.0 / 13.0)
#define ORC_SMAX 250

/* RKC coefficients for s stages, Section 2.3. Arrays of length s+1, index j.
 * mu[j], nu[j], mut[j] (mu~), gt[j] (gamma~) for j >= 2, mut[1] = mu~_1.
 * Also returns w0, w1 and the stage abscissae c[j] (0..s). */
void orc_rkc_coeffs(int s, double *mu, double *nu, double *mut, double *gt,
                    double *c, double *w0_out, double *w1_out)
{
    double *T = (double *)xmalloc(sizeof(double) * 6 * (s + 1));
    double *dT = T + (s + 1), *ddT = dT + (s + 1), *b = ddT + (s + 1), *a = b + (s + 1);
    double w0 = 1.0 + ORC_KAPPA / ((double)s * s), w1;
    int j;
    T[0] = 1.0; dT[0] = 0.0; ddT[0] = 0.0;
    T[1] = w0;  dT[1] = 1.0; ddT[1] = 0.0;
    for (j = 2; j <= s; j++) {
        T[j] = 2.0 * w0 * T[j - 1] - T[j - 2];
        dT[j] = 2.0 * T[j - 1] + 2.0 * w0 * dT[j - 1] - dT[j - 2];
        ddT[j] = 4.0 * dT[j - 1] + 2.0 * w0 * ddT[j - 1] - ddT[j - 2];
    }
    w1 = dT[s] / ddT[s];
    for (j = 2; j <= s; j++) b[j] = ddT[j] / (dT[j] * dT[j]);
    b[0] = b[2];
    b[1] = b[2];
    for (j = 0; j <= s; j++) a[j] = 1.0 - b[j] * T[j];
    mu[0] = nu[0] = mut[0] = gt[0] = 0.0;
    mu[1] = nu[1] = gt[1] = 0.0;
    mut[1] = b[1] * w1;
    for (j = 2; j <= s; j++) {
        mu[j] = 2.0 * b[j] * w0 / b[j - 1];
        nu[j] = -b[j] / b[j - 2];
        mut[j] = 2.0 * b[j] * w1 / b[j - 1];
        gt[j] = -a[j - 1] * mut[j];
    }
    if (c) {
        c[0] = 0.0;
        for (j = 2; j < s; j++) c[j] = w1 * ddT[j] / dT[j];
        c[s] = 1.0;
        c[1] = (s > 2 ? c[2] : w1 * ddT[2] / dT[2]) / dT[2];
    }
    if (w0_out) *w0_out = w0;
    if (w1_out) *w1_out = w1;
    free(T);
}

/* One s-stage RKC step of size h from y with f0 = f(y), Eqs. (E:rkc0)-(E:rkcs).
 * ys: output w_s. wk: 3*n doubles. */
static void rkc_step(orc_f *F, int n, const double *y, const double *f0, double h, int s,
                     double *ys, double *wk)
{
    double *mu = (double *)xmalloc(sizeof(double) * 4 * (s + 1));
    double *nu = mu + (s + 1), *mut = nu + (s + 1), *gt = mut + (s + 1);
    double *wm2 = wk, *wm1 = wk + n, *fj = wk + 2 * n; /* w_{j-2}, w_{j-1}, f_{j-1} */
    int i, j;
    orc_rkc_coeffs(s, mu, nu, mut, gt, NULL, NULL, NULL);
    for (i = 0; i < n; i++) {
        wm2[i] = y[i];
        wm1[i] = y[i] + mut[1] * h * f0[i];
    }
    for (j = 2; j <= s; j++) {
        feval(F, wm1, fj);
        for (i = 0; i < n; i++) {
            double wj = (1.0 - mu[j] - nu[j]) * y[i] + mu[j] * wm1[i] + nu[j] * wm2[i]
                        + mut[j] * h * fj[i] + gt[j] * h * f0[i];
            wm2[i] = wm1[i];
            wm1[i] = wj;
        }
    }
    memcpy(ys, wm1, sizeof(double) * n);
    free(mu);
}

/* Eq. (E:rmsE): || Delta / (T sqrt(N)) ||_2 with T_i = atol + rtol max(|a_i|,|b_i|). */
static double rms_norm(int n, const double *d, const double *ya, const double *yb,
                       double rtol, double atol)
{
    double acc = 0.0;
    int i;
    for (i = 0; i < n; i++) {
        double sc = atol + rtol * fmax(fabs(ya[i]), fabs(yb[i]));
        double r = d[i] / sc;
        acc += r * r;
    }
    return sqrt(acc / n);
}

/* Gershgorin bound on a forward-difference Jacobian at y (f0 = f(y)). */
static double gershgorin(orc_f *F, int n, const double *y, const double *f0, double atol,
                         double *x, double *fx, double *rowsum)
{
    const double sqrt_u = sqrt(ldexp(1.0, -52));
    double sigma = 0.0;
    int i, k;
    for (i = 0; i < n; i++) rowsum[i] = 0.0;
    for (k = 0; k < n; k++) {
        double eps = sqrt_u * fmax(fabs(y[k]), atol);
        memcpy(x, y, sizeof(double) * n);
        x[k] = y[k] + eps;
        feval(F, x, fx);
        for (i = 0; i < n; i++) rowsum[i] += fabs((fx[i] - f0[i]) / eps);
    }
    for (i = 0; i < n; i++) if (rowsum[i] > sigma) sigma = rowsum[i];
    return sigma;
}

/* Nonlinear power method for the spectral radius (the paper's choice, end of
 * Section 2.3): repeated finite-difference products w = f(y + v) - f(y) ~ J v
 * with v rescaled to length dyn = sqrt(u) ||y||_2 (sqrt(u) if y = 0), starting
 * from the warm-start direction v (the previous estimate's eigenvector; f(y)
 * at the first estimate; all ones if that is zero). The estimate ||w||/dyn is
 * accepted once two successive values agree to 1 % (at most 20 products) and
 * returned with a 20 % margin, since the iteration approaches |lambda_max|
 * from below. v is left holding the new direction. *iters receives the
 * number of f evaluations. */
static double power_sigma(orc_f *F, int n, const double *y, const double *f0, double *v,
                          double *z, double *fz, int *iters)
{
    const double sqrt_u = sqrt(ldexp(1.0, -52));
    double ynorm = 0.0, vnorm = 0.0, dyn, sig = 0.0, prev = 0.0;
    int i, k;
    for (i = 0; i < n; i++) ynorm += y[i] * y[i];
    ynorm = sqrt(ynorm);
    dyn = ynorm > 0.0 ? sqrt_u * ynorm : sqrt_u;
    for (i = 0; i < n; i++) vnorm += v[i] * v[i];
    vnorm = sqrt(vnorm);
    if (!(vnorm > 0.0) || !isfinite(vnorm)) {
        for (i = 0; i < n; i++) v[i] = 1.0;
        vnorm = sqrt((double)n);
    }
    for (i = 0; i < n; i++) v[i] *= dyn / vnorm;
    *iters = 0;
    for (k = 1; k <= 20; k++) {
        double wnorm = 0.0;
        for (i = 0; i < n; i++) z[i] = y[i] + v[i];
        feval(F, z, fz);
        (*iters)++;
        for (i = 0; i < n; i++) {
            fz[i] -= f0[i];
            wnorm += fz[i] * fz[i];
        }
        wnorm = sqrt(wnorm);
        sig = wnorm / dyn;
        if (!(wnorm > 0.0) || !isfinite(wnorm)) break;
        for (i = 0; i < n; i++) v[i] = fz[i] * (dyn / wnorm);
        if (k >= 2 && fabs(sig - prev) <= 0.01 * sig) break;
        prev = sig;
    }
    return 1.2 * sig;
}

double orc_sigma_power(const void *mp, double T, double p, const double *y, double *v,
                       int32_t *iters)
{
    const orc_mech *m = (const orc_mech *)mp;
    int n = m->nS, it = 0;
    double *k = (double *)xmalloc(sizeof(double) * 2 * m->nR);
    double *work = (double *)xmalloc(sizeof(double) * (2 * m->nS + 2 * m->nR));
    double *w = (double *)xmalloc(sizeof(double) * 3 * n);
    orc_f F;
    double sigma;
    orc_rate_constants(m, T, k, k + m->nR);
    F.m = m; F.T = T; F.p = p; F.k = k; F.k0 = k + m->nR; F.work = work; F.energy = 0; F.nfe = 0;
    feval(&F, y, w);
    sigma = power_sigma(&F, n, y, w, v, w + n, w + 2 * n, &it);
    *iters = it;
    free(k); free(work); free(w);
    return sigma;
}

double orc_sigma(const void *mp, double T, double p, const double *y, double atol)
{
    const orc_mech *m = (const orc_mech *)mp;
    int n = m->nS;
    double *k = (double *)xmalloc(sizeof(double) * 2 * m->nR);
    double *work = (double *)xmalloc(sizeof(double) * (2 * m->nS + 2 * m->nR));
    double *v = (double *)xmalloc(sizeof(double) * 4 * n);
    orc_f F;
    double sigma;
    orc_rate_constants(m, T, k, k + m->nR);
    F.m = m; F.T = T; F.p = p; F.k = k; F.k0 = k + m->nR; F.work = work; F.energy = 0; F.nfe = 0;
    feval(&F, y, v);
    sigma = gershgorin(&F, n, y, v, atol, v + n, v + 2 * n, v + 3 * n);
    free(k); free(work); free(v);
    return sigma;
}

static int rkc_stages(double h, double sigma)
{
    double s = floor(1.0 + sqrt(1.0 + 1.54 * h * sigma));
    if (s < 2.0) return 2;
    if (s > ORC_SMAX) return ORC_SMAX + 1; /* caller caps */
    return (int)s;
}

/* sigma by the selected estimator: 1 Gershgorin on the FD Jacobian,
 * 2 nonlinear power method with warm start in ev */
static double estimate_sigma(orc_f *F, int n, int est, const double *y, const double *f0,
                             double atol, double *x, double *fx, double *rowsum, double *ev)
{
    int it;
    if (est == 2) return power_sigma(F, n, y, f0, ev, x, fx, &it);
    return gershgorin(F, n, y, f0, atol, x, fx, rowsum);
}

static int rkc_cell(orc_f *F, int n, double *y, double dt, double rtol, double atol,
                    int max_steps, orc_stats *st, int est)
{
    double *v = (double *)xmalloc(sizeof(double) * n * 10);
    double *f0 = v, *x = v + n, *fx = v + 2 * n, *ys = v + 3 * n, *d = v + 4 * n;
    double *wk = v + 5 * n, *rowsum = v + 8 * n, *ev = v + 9 * n;
    double t = 0.0, hmin = 1e-20 * dt, sigma, h, h0, e0, err_prev = 0.0, h_prev = 0.0;
    int i, status = 0, attempts = 0, since_sigma = 0, sigma_here, last_rejected = 0;
    int have_prev = 0;
    long nfe0;

    feval(F, y, f0);
    if (!all_finite(n, f0)) { free(v); return 3; }
    memcpy(ev, f0, sizeof(double) * n); /* first power-method direction */
    nfe0 = F->nfe;
    sigma = estimate_sigma(F, n, est, y, f0, atol, x, fx, rowsum, ev);
    st->nfs += (int)(F->nfe - nfe0);
    st->nsig++;
    sigma_here = 1;
    if (!isfinite(sigma)) { free(v); return 3; }

    /* initial step, Section 2.3: h0 = 1/sigma, Delta_0 = h0 (f(y0 + h0 f0) - f0),
     * h1 = 0.1 h0 / ||Delta_0||^{1/2} */
    h0 = sigma > 0.0 ? 1.0 / sigma : dt;
    if (h0 > dt) h0 = dt;
    for (i = 0; i < n; i++) x[i] = y[i] + h0 * f0[i];
    feval(F, x, fx);
    for (i = 0; i < n; i++) d[i] = h0 * (fx[i] - f0[i]);
    e0 = rms_norm(n, d, y, y, rtol, atol);
    if (!isfinite(e0))
        h = 0.1 * h0;
    else
        h = e0 > 0.0 ? 0.1 * h0 / sqrt(e0) : dt;
    if (h > dt) h = dt;
    if (h < hmin) { free(v); return 2; }

    for (;;) {
        double hh = h, err, fac;
        int s, last = 0;
        if (attempts >= max_steps) { status = 1; break; }
        if (since_sigma >= 25 || (last_rejected && !sigma_here)) {
            nfe0 = F->nfe;
            sigma = estimate_sigma(F, n, est, y, f0, atol, x, fx, rowsum, ev);
            st->nfs += (int)(F->nfe - nfe0);
            st->nsig++;
            since_sigma = 0;
            sigma_here = 1;
            if (!isfinite(sigma)) { status = 3; break; }
        }
        if (hh >= dt - t) { hh = dt - t; last = 1; }
        s = rkc_stages(hh, sigma);
        if (s > ORC_SMAX) {
            s = ORC_SMAX;
            hh = ((ORC_SMAX - 1.0) * (ORC_SMAX - 1.0) - 1.0) / (1.54 * sigma);
            last = 0;
        }
        rkc_step(F, n, y, f0, hh, s, ys, wk);
        feval(F, ys, fx);
        attempts++;
        for (i = 0; i < n; i++) d[i] = 0.8 * (y[i] - ys[i]) + 0.4 * hh * (f0[i] + fx[i]);
        err = rms_norm(n, d, y, ys, rtol, atol);
        trace(st, hh, err, s, err <= 1.0, sigma);
        if (err <= 1.0) {
            st->nacc++;
            if (err == 0.0)
                fac = 10.0;
            else if (have_prev && !last_rejected && err_prev > 0.0)
                fac = 0.8 * (hh / h_prev) * cbrt(err_prev) / pow(err, 2.0 / 3.0);
            else
                fac = 0.8 / cbrt(err);
            if (fac > 10.0) fac = 10.0;
            if (fac < 0.1) fac = 0.1;
            memcpy(y, ys, sizeof(double) * n);
            memcpy(f0, fx, sizeof(double) * n);
            t = last ? dt : t + hh;
            if (last) break;
            have_prev = 1;
            h_prev = hh;
            err_prev = err;
            last_rejected = 0;
            sigma_here = 0;
            since_sigma++;
            h = fac * hh;
        } else {
            /* err > 1 or not finite (the trial step blew up): reject */
            st->nrej++;
            fac = isfinite(err) ? 0.8 / cbrt(err) : 0.1;
            if (fac < 0.1) fac = 0.1;
            last_rejected = 1;
            h = fac * hh;
            if (h < hmin) { status = 2; break; }
        }
    }
    free(v);
    return status;
}

/* Single-step entry points for tests (no step control). */
void orc_rkck_single(const void *mp, double T, double p, const double *y, double h,
                     double *y5, double *err)
{
    const orc_mech *m = (const orc_mech *)mp;
    int n = m->nS;
    double *k = (double *)xmalloc(sizeof(double) * 2 * m->nR);
    double *work = (double *)xmalloc(sizeof(double) * (2 * m->nS + 2 * m->nR));
    double *v = (double *)xmalloc(sizeof(double) * 8 * n);
    orc_f F;
    orc_rate_constants(m, T, k, k + m->nR);
    F.m = m; F.T = T; F.p = p; F.k = k; F.k0 = k + m->nR; F.work = work; F.energy = 0; F.nfe = 0;
    feval(&F, y, v);
    rkck_step(&F, n, y, v, h, y5, err, v + 2 * n, v + n);
    free(k); free(work); free(v);
}

void orc_rkc_single(const void *mp, double T, double p, const double *y, double h, int s,
                    double *ys)
{
    const orc_mech *m = (const orc_mech *)mp;
    int n = m->nS;
    double *k = (double *)xmalloc(sizeof(double) * 2 * m->nR);
    double *work = (double *)xmalloc(sizeof(double) * (2 * m->nS + 2 * m->nR));
    double *v = (double *)xmalloc(sizeof(double) * 4 * n);
    orc_f F;
    orc_rate_constants(m, T, k, k + m->nR);
    F.m = m; F.T = T; F.p = p; F.k = k; F.k0 = k + m->nR; F.work = work; F.energy = 0; F.nfe = 0;
    feval(&F, y, v);
    rkc_step(&F, n, y, v, h, s, ys, v + n);
    free(k); free(work); free(v);
}

/* Integrate `cells` independent cells over dt. Y is species-major,
 * Y[i * ldY + cell]; it is updated in place. method 0 = RKCK, 1 = RKC with
 * the Gershgorin spectral radius, 2 = RKC with the power-method one.
 * energy != 0 integrates T with the energy equation as the (nS+1)-th
 * component and writes it back to Tc (the mechanism needs thermochemistry;
 * without it nothing is done and -1 is returned).
 * Per-cell outputs (any may be NULL): status, and stats[cell] =
 * {f evaluations, accepted steps, rejected steps, sigma estimates, f
 * evaluations inside the sigma estimates}.
 * Returns the number of threads used.
 * nthreads > 0 sets the OpenMP thread count when built with OpenMP
 * (<= 0: all available threads). */
int orc_integrate(const void *mp, int64_t cells, double *Tc, const double *pc,
                  double *Y, int64_t ldY, double dt, double rtol, double atol, int method,
                  int max_steps, uint8_t *status, int32_t *stats, int nthreads, int energy)
{
    const orc_mech *m = (const orc_mech *)mp;
    int64_t c;
    int nt = 1;
    if (energy && !m->cp) return -1;
    if (max_steps <= 0) max_steps = 100000;
#ifdef _OPENMP
    nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
#endif
    for (c = 0; c < cells; c++) {
        int n = m->nS + (energy ? 1 : 0), i, st;
        double *y = (double *)xmalloc(sizeof(double) * n);
        double *k = (double *)xmalloc(sizeof(double) * 2 * m->nR);
        double *work = (double *)xmalloc(sizeof(double) * (2 * m->nS + 2 * m->nR));
        orc_stats S = {0, 0, 0, 0, 0, 0, 0, NULL, NULL, NULL, NULL, NULL};
        orc_f F;
        for (i = 0; i < m->nS; i++) y[i] = Y[(int64_t)i * ldY + c];
        if (energy) y[m->nS] = Tc[c];
        orc_rate_constants(m, Tc[c], k, k + m->nR);
        F.m = m; F.T = Tc[c]; F.p = pc[c]; F.k = k; F.k0 = k + m->nR; F.work = work;
        F.energy = energy; F.nfe = 0;
        if (method == 0)
            st = rkck_cell(&F, n, y, dt, rtol, atol, max_steps, &S);
        else
            st = rkc_cell(&F, n, y, dt, rtol, atol, max_steps, &S, method);
        for (i = 0; i < m->nS; i++) Y[(int64_t)i * ldY + c] = y[i];
        if (energy) Tc[c] = y[m->nS];
        if (status) status[c] = (uint8_t)st;
        if (stats) {
            stats[5 * c + 0] = (int32_t)F.nfe;
            stats[5 * c + 1] = S.nacc;
            stats[5 * c + 2] = S.nrej;
            stats[5 * c + 3] = S.nsig;
            stats[5 * c + 4] = S.nfs;
        }
        free(y); free(k); free(work);
    }
    return nt;
}

/* One cell with a per-attempt trace of at most cap entries. Returns the cell
 * status; *len receives the number of attempts (may exceed cap) and stats
 * (if not NULL) the cell's five counters as in orc_integrate. tr_sig may be
 * NULL. With energy != 0, y holds nS + 1 components, T last (T is ignored). */
int orc_trace_cell(const void *mp, double T, double p, double *y, double dt, double rtol,
                   double atol, int method, int max_steps, int cap, double *tr_h,
                   double *tr_err, int32_t *tr_s, int32_t *tr_acc, int32_t *len, int energy,
                   double *tr_sig, int32_t *stats)
{
    const orc_mech *m = (const orc_mech *)mp;
    int n = m->nS + (energy ? 1 : 0), st;
    double *k = (double *)xmalloc(sizeof(double) * 2 * m->nR);
    double *work = (double *)xmalloc(sizeof(double) * (2 * m->nS + 2 * m->nR));
    orc_stats S = {0, 0, 0, 0, 0, cap, 0, tr_h, tr_err, tr_sig, (int *)tr_s, (int *)tr_acc};
    orc_f F;
    if (energy && !m->cp) { free(k); free(work); return -1; }
    if (max_steps <= 0) max_steps = 100000;
    if (energy) T = y[m->nS];
    orc_rate_constants(m, T, k, k + m->nR);
    F.m = m; F.T = T; F.p = p; F.k = k; F.k0 = k + m->nR; F.work = work;
    F.energy = energy; F.nfe = 0;
    st = method == 0 ? rkck_cell(&F, n, y, dt, rtol, atol, max_steps, &S)
                     : rkc_cell(&F, n, y, dt, rtol, atol, max_steps, &S, method);
    *len = S.len;
    if (stats) {
        stats[0] = (int32_t)F.nfe;
        stats[1] = S.nacc;
        stats[2] = S.nrej;
        stats[3] = S.nsig;
        stats[4] = S.nfs;
    }
    free(k); free(work);
    return st;
}

int orc_has_openmp(void)
{
#ifdef _OPENMP
    return 1;
#else
    return 0;
#endif
}
