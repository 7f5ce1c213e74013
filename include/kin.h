/*
 * kin.h -- C ABI of the GB300 batched chemical-kinetics integrator.
 *
 * The library integrates many independent per-cell kinetics systems
 * dY/dt = f(T, p, Y) over one operator-split flow step dt. The integration
 * restarts every call, with internal sub-stepping and no memory between calls
 * (Niemeyer & Sung, Section 3). Two methods are available:
 *   KIN_RKCK  Runge-Kutta-Cash-Karp 5(4), Section 2.2, Table 1, Eq. (E:hnew);
 *   KIN_RKC   second-order Runge-Kutta-Chebyshev, Section 2.3, Eqs.
 *             (E:rkc0)-(E:rkcs), (E:rmsE). The spectral radius is a Gershgorin
 *             bound on a finite-difference Jacobian or, as in the paper, a
 *             nonlinear power method (kin_opts.sigma).
 * f is the species source term of Section 2.1, Eqs. (E:mass), (E:spec-rate),
 * (E:rxn-rate) and (E:rxn-const), with third-body and Lindemann falloff
 * reactions. By default temperature and pressure are held fixed over the flow
 * step, so N = n_species. With kin_opts.energy the constant-pressure energy
 * equation of Section 2.1, Eq. (E:energy), is integrated too (N = n_species +
 * 1): T changes and is written back, and k_j, density and concentrations follow
 * it at every evaluation of f.
 *
 * Conventions for every entry point:
 *  - Device pointers are CUDA device memory of the current device; host
 *    pointers are ordinary host memory. Nothing is retained after a call
 *    returns except inside a kin_mech.
 *  - State layout is species-major: Y[i * ldY + c] holds species i of cell c,
 *    with ldY >= cells.
 *  - Units: T in K, p in Pa, Y as mass fractions, dt in s, W in g/mol,
 *    A in cm-mol-s units (given as ln A), Ea in J/mol.
 *  - Work is enqueued on opts->stream (a cudaStream_t; NULL means the legacy
 *    default stream). Calls return before the GPU finishes; results, per-cell
 *    status and statistics are valid after the stream is synchronised.
 *  - Return value: KIN_OK, or a negative KIN_E* code. kin_last_error() then
 *    describes the failure (thread-local, valid until the next call on the
 *    same thread). A failed call enqueues no work.
 *  - A cell that cannot finish does not fail the call; its status byte says
 *    why and its Y holds the last accepted state (see KIN_CELL_*).
 */
#ifndef KIN_H
#define KIN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define KIN_OK 0
#define KIN_EINVAL (-1)       /* bad argument: null pointer, size, non-finite or non-positive dt/tol */
#define KIN_ENOMEM (-2)       /* device or host allocation failed, or workspace too small */
#define KIN_ECUDA (-3)        /* a CUDA call failed (message has the CUDA error string) */
#define KIN_EUNSUPPORTED (-4) /* mechanism or option combination not supported */

/* method */
#define KIN_RKCK 0
#define KIN_RKC 1
/* precision: FP64 everywhere, or FP32 rate evaluation (Arrhenius exp and
 * rate-of-progress products, stoichiometric sum) with FP64 state, stage
 * accumulation, error norm, step control and spectral-radius bound. */
#define KIN_FP64 0
#define KIN_MIXED 1

/* staging of the per-lane rate scratch */
#define KIN_STAGE_GLOBAL 0     /* every per-lane array in the workspace */
#define KIN_STAGE_SHARED 1     /* concentrations and rates of progress in shared memory */
#define KIN_STAGE_SHARED_ALL 2 /* ... and the cell's rate constants too */

/* RKC spectral-radius estimator */
#define KIN_SIGMA_GERSHGORIN 0
#define KIN_SIGMA_POWER 1

/* kernel register budget */
#define KIN_OCC_DEFAULT 0
#define KIN_OCC_HIGH 1

/* work decomposition across the GPU's lanes */
#define KIN_LAYOUT_AUTO 0 /* library choice: KIN_LAYOUT_WARP when n_reactions >
                             KIN_WARP_MIN_REACTIONS or the call has fewer than
                             KIN_WARP_MAX_CELLS_PER_SM cells per SM of the device (too
                             few to give every lane a cell), else KIN_LAYOUT_LANE */
#define KIN_LAYOUT_LANE 1 /* one lane integrates one cell (the paper's thread-per-ODE
                             design, Section 3): per-cell arrays in the workspace or in
                             shared memory (kin_opts.staging) */
#define KIN_LAYOUT_WARP 2 /* one warp integrates one cell: its 32 lanes share the
                             reactions and species of f; the cell's concentrations and
                             rates of progress live in shared memory. staging is
                             ignored; for RKC, occupancy selects the register budget
                             (KIN_OCC_HIGH: for up to 64 state components 48
                             registers and 40 warps per SM, or 80 registers and 24
                             warps with the energy equation); block_threads may be up
                             to 256 */
#define KIN_WARP_MIN_REACTIONS 256
#define KIN_WARP_MAX_CELLS_PER_SM 64

/* how the lane-per-cell layout evaluates f (kin_opts.feval) */
#define KIN_FEVAL_AUTO 0      /* the generated f for an isothermal call of at least
                                 KIN_GEN_MIN_CELLS cells that it serves (below), else the
                                 tables: the one-time compilation pays for itself on large
                                 calls (with the energy equation the generated form, one
                                 inlined exp per reaction, is slower than the tables) */
#define KIN_FEVAL_TABLE 1     /* one kernel for every mechanism: f reads the mechanism's
                                 device tables, its concentrations and rates of progress
                                 sit in per-lane arrays */
#define KIN_FEVAL_GENERATED 2 /* f for this mechanism as straight-line FP64 code (species
                                 indices, efficiencies and coefficients as literals,
                                 concentrations and production rates in registers),
                                 compiled with NVRTC on first use and cached per device and
                                 mechanism; with the energy equation too (the rate
                                 constants then follow T inside f). Serves KIN_FP64,
                                 KIN_LAYOUT_LANE, KIN_STAGE_GLOBAL and mechanisms of at most
                                 KIN_GEN_MAX_SPECIES species and KIN_GEN_MAX_REACTIONS
                                 reactions; KIN_EUNSUPPORTED otherwise or without NVRTC,
                                 KIN_ECUDA if the compilation fails. The first such call
                                 of a mechanism compiles and loads f on the host: make it
                                 before capturing the call into a CUDA graph */
#define KIN_GEN_MAX_SPECIES 32
#define KIN_GEN_MAX_REACTIONS 256
#define KIN_GEN_MIN_CELLS 65536

/* per-cell status */
#define KIN_CELL_OK 0
#define KIN_CELL_MAXSTEPS 1  /* attempted-step limit reached */
#define KIN_CELL_HMIN 2      /* step size fell below 1e-20 * dt */
#define KIN_CELL_NONFINITE 3 /* f (or the RKC spectral-radius bound) is not finite at
                                the initial or an accepted state */

/* reaction types */
#define KIN_RXN_PLAIN 0
#define KIN_RXN_THIRD_BODY 1 /* Omega = k [M] prod C,   [M] = sum_k eff_k C_k */
#define KIN_RXN_FALLOFF 2    /* Lindemann: Omega = k_inf Pr/(1+Pr) prod C, Pr = k_0 [M] / k_inf */

/* Host description of an irreversible mechanism. Caller-owned; copied by
 * kin_create_mechanism. Each reaction has up to two reactants and two products
 * (index -1 marks an empty slot; a species listed twice has coefficient 2). */
typedef struct {
    int32_t n_species;   /* >= 1, <= KIN_MAX_SPECIES */
    int32_t n_reactions; /* >= 0, <= KIN_MAX_REACTIONS */
    const double *W;     /* [n_species] molar masses, > 0 */
    const double *lnA;   /* [n_reactions] ln of the pre-exponential factor */
    const double *beta;  /* [n_reactions] temperature exponent */
    const double *Ea;    /* [n_reactions] activation energy, J/mol */
    const int32_t *reac; /* [n_reactions][2] reactant species or -1 */
    const int32_t *prod; /* [n_reactions][2] product species or -1 */
    const int8_t *type;  /* [n_reactions] KIN_RXN_* */
    const double *eff;   /* [n_rows][n_species] third-body efficiencies, one row
                            per non-plain reaction in reaction order; may be NULL
                            when every reaction is plain */
    const double *lnA0;  /* [n_reactions] low-pressure limit of falloff reactions */
    const double *beta0; /* (read only where type == KIN_RXN_FALLOFF; the three */
    const double *Ea0;   /*  may be NULL when there is none) */
    const double *cp;    /* [n_species] molar heat capacity at constant pressure,
                            J/(mol K), > 0; and */
    const double *Hf;    /* [n_species] formation enthalpy at 298.15 K, J/mol: the
                            species enthalpy is H_i(T) = Hf_i + cp_i (T - 298.15).
                            Both NULL when the energy equation is not needed */
} kin_mech_desc;

#define KIN_MAX_SPECIES 256
#define KIN_MAX_REACTIONS 8192
#define KIN_MAX_STAGES 250 /* RKC stage cap */

typedef struct kin_mech kin_mech; /* opaque: device-resident tables */

typedef struct {
    int32_t method;        /* KIN_RKCK or KIN_RKC */
    int32_t precision;     /* KIN_FP64 or KIN_MIXED */
    int32_t max_steps;     /* attempted steps per cell; <= 0 means 100000 */
    int32_t block_threads; /* threads per block, multiple of 32, <= 128 (<= 256 with
                              KIN_LAYOUT_WARP); 0 = library choice (128) */
    int32_t blocks_per_sm; /* persistent blocks per SM; 0 = as many as fit (lane layout:
                              <= 512 threads per SM, 768 with KIN_OCC_HIGH) */
    int32_t staging;       /* KIN_STAGE_*: where f's per-lane arrays live. Shared staging
                              needs (n_species + n_reactions) [+ n_reactions + n_falloff
                              for SHARED_ALL] x block_threads elements of the rate type
                              per block; KIN_EUNSUPPORTED if that does not fit */
    int32_t occupancy;     /* KIN_OCC_DEFAULT: kernel built for up to 16 resident warps per
                              SM; KIN_OCC_HIGH: built with a register cap for 24 (the
                              warp layout's caps are listed with KIN_LAYOUT_WARP) */
    int32_t sigma;         /* RKC spectral radius: KIN_SIGMA_GERSHGORIN (Gershgorin bound on a
                              finite-difference Jacobian, n_species f evaluations) or
                              KIN_SIGMA_POWER (nonlinear power method with warm start, the
                              paper's choice, end of Section 2.3); ignored for RKCK */
    int32_t layout;        /* KIN_LAYOUT_*: one lane or one warp per cell. Both give the
                              same method, decisions and statistics up to the rounding
                              order of sums (results agree within the integration
                              tolerance, not bit for bit) */
    int32_t energy;        /* 0: T fixed over the flow step. 1: integrate the energy
                              equation, Eq. (E:energy): dT/dt = -(1/(rho cp)) sum_i
                              h_i omega_i W_i with cp = sum_i Y_i cp_i / W_i; T is part
                              of the state (error norm, spectral radius) and is
                              written back to T. Needs the mechanism's cp and Hf
                              (else KIN_EUNSUPPORTED) */
    int32_t feval;         /* KIN_FEVAL_*: tables or generated f (lane layout). Both follow
                              the same method and decisions; the generated f rounds its
                              sums in another order (results agree within the
                              integration tolerance, not bit for bit) */
    void *stream;          /* cudaStream_t */
} kin_opts;

/* One independent group of cells ("instance") of a batched call. All pointers
 * are device pointers with the layouts described above. */
typedef struct {
    int64_t cells;     /* >= 0 */
    double *T;         /* [cells]; updated in place with opts->energy, else read only */
    const double *p;   /* [cells] */
    double *Y;         /* [n_species][ldY], updated in place */
    int64_t ldY;       /* >= cells */
    double dt, rtol, atol; /* dt > 0, rtol > 0, atol >= 0, all finite */
    uint8_t *status;   /* [cells] KIN_CELL_*, or NULL */
    int32_t *stats;    /* [cells][KIN_NSTATS]: f evaluations, accepted steps,
                          rejected steps, spectral-radius estimates, and the f
                          evaluations spent inside those estimates (part of the
                          first count); or NULL */
} kin_instance;

#define KIN_MAX_INSTANCES 128
#define KIN_NSTATS 5 /* statistics per cell */

/* Copy and validate a mechanism, upload its tables to the current device and
 * precompute the RKC coefficient table there (Section 2.3, s = 2..250).
 * Synchronous. Errors: KIN_EINVAL (null desc/out, sizes out of range, species
 * index out of range, W <= 0, non-finite parameter, missing efficiency rows),
 * KIN_ENOMEM, KIN_ECUDA. */
int kin_create_mechanism(const kin_mech_desc *desc, kin_mech **out);

/* Free a mechanism. cudaFree waits for outstanding work on the device; do
 * not destroy a mechanism that a captured CUDA graph still uses. NULL is a
 * no-op. */
int kin_destroy(kin_mech *m);

/* Message for the last failed call on this thread ("" if none). */
const char *kin_last_error(void);

/* Bytes of device workspace that kin_integrate / kin_integrate_batch (with
 * `cells` cells in total) or kin_rates (with `cells` cells) need for `opts` on
 * the current device: per-lane working vectors of the persistent grid plus
 * per-cell rate constants, f(y0), first-step data and processing order.
 * Returns < 0 on error. */
int64_t kin_workspace_bytes(const kin_mech *m, const kin_opts *opts, int64_t cells);

/* Integrate `cells` cells of one instance over dt (Sections 2.2/2.3 and the
 * restart-per-flow-step convention of Section 3). T, p, Y, status, stats
 * as in kin_instance. workspace: caller-owned device memory of at least
 * kin_workspace_bytes(m, opts, cells) bytes, 256-byte aligned; it must not be
 * used by another call that may run concurrently. Errors: KIN_EINVAL, KIN_ENOMEM
 * (workspace too small), KIN_EUNSUPPORTED, KIN_ECUDA. */
int kin_integrate(const kin_mech *m, int64_t cells, double *T, const double *p,
                  double *Y, int64_t ldY, double dt, double rtol, double atol,
                  const kin_opts *opts, uint8_t *status, int32_t *stats,
                  void *workspace, int64_t workspace_bytes);

/* Integrate up to KIN_MAX_INSTANCES instances (each with its own cells, dt and
 * tolerances) in one persistent launch; lanes take cells from a shared queue,
 * so uneven instances balance across the GPU. `inst` is a host array that is
 * copied into the launch parameters, so the call may be captured in a CUDA
 * graph (the captured graph refers to the same device buffers and workspace).
 * The workspace must hold kin_workspace_bytes(m, opts, total cells). Errors
 * as kin_integrate. */
int kin_integrate_batch(const kin_mech *m, int32_t n_instances, const kin_instance *inst,
                        const kin_opts *opts, void *workspace, int64_t workspace_bytes);

/* Device bytes kin_integrate_host needs for `cells` cells (its staging
 * copies of T, p, Y, status and stats plus the workspace). < 0 on error. */
int64_t kin_host_buffer_bytes(const kin_mech *m, const kin_opts *opts, int64_t cells);

/* Host-buffer form of kin_integrate, for callers whose state lives in host
 * memory: T, p, Y (in/out), status and stats are HOST pointers with the
 * layouts above (status and stats may be NULL). On opts->stream the call
 * copies T, p and Y into `device_buffer` (device memory of at least
 * kin_host_buffer_bytes bytes, 256-byte aligned), integrates there, and copies
 * Y (and T with opts->energy), status and stats back. Page-locked host memory makes every copy
 * asynchronous; with pageable memory the copies may block. Host results are
 * valid after the stream is synchronised. Errors as kin_integrate. */
int kin_integrate_host(const kin_mech *m, int64_t cells, double *T, const double *p,
                       double *Y, int64_t ldY, double dt, double rtol, double atol,
                       const kin_opts *opts, uint8_t *status, int32_t *stats,
                       void *device_buffer, int64_t device_bytes);

/* Size of the fixed device array behind kin_integrate_noalloc (64 MiB). */
#define KIN_NOALLOC_SCRATCH_BYTES (64ull << 20)

/* kin_integrate for callers that cannot allocate device memory when they
 * integrate (for example a flow solver whose own memory manager owns the
 * device, or code running where allocation is not allowed). Same arguments,
 * meaning and errors as kin_integrate, minus the workspace: the working memory
 * comes from a fixed array of KIN_NOALLOC_SCRATCH_BYTES that the library
 * reserves on every device where it is used and keeps until the process
 * exits. After its first call on a device, the call allocates nothing.
 *  - The first call on a device loads that array (64 MiB of device memory)
 *    and looks up its device address with the device current: make it at
 *    start-up, before any stream capture. If the device has no room for the
 *    array, that call fails with KIN_ENOMEM.
 *  - The array is shared by all calls on a device and keeps the last call's
 *    contents; each call clears what must start at zero. Calls that overlap
 *    on the GPU (on different streams, or from different threads) race on it:
 *    serialise them.
 *  - The working memory grows with the cell count and the persistent blocks
 *    per SM. blocks_per_sm is resolved as in kin_integrate (0: as many as
 *    fit); when that workspace exceeds the array, the call steps down to the
 *    largest count that fits. A call that does not fit even at one block per
 *    SM (for a 13-species / 54-reaction mechanism in FP64 on a 152-SM GPU,
 *    about 57,000 cells) fails with KIN_ENOMEM and launches nothing.
 *  - It never compiles a generated f (KIN_FEVAL_GENERATED), because the
 *    compilation and the library load allocate. With KIN_FEVAL_AUTO it uses
 *    the tables unless an earlier call loaded the mechanism's generated f on
 *    this device (then it chooses as kin_integrate does); KIN_FEVAL_GENERATED
 *    fails with KIN_EUNSUPPORTED until such a call has loaded it.
 * The paper has no counterpart of this entry point. */
int kin_integrate_noalloc(const kin_mech *m, int64_t cells, double *T, const double *p,
                          double *Y, int64_t ldY, double dt, double rtol, double atol,
                          const kin_opts *opts, uint8_t *status, int32_t *stats);

/* f alone: dYdt[i * ldY + c] = f(T_c, p_c, Y_c)_i (Eqs. (E:mass),
 * (E:spec-rate), (E:rxn-rate), (E:rxn-const)) in the given precision
 * (KIN_FP64 or KIN_MIXED), enqueued on `stream`. T, p, Y, dYdt and workspace
 * are device pointers; dYdt has the layout of Y. The workspace rule is that of
 * kin_integrate with method KIN_RKC, the same precision, layout
 * KIN_LAYOUT_LANE, default launch shape and `cells` cells. Errors:
 * KIN_EINVAL, KIN_ENOMEM, KIN_ECUDA. */
int kin_rates(const kin_mech *m, int64_t cells, const double *T, const double *p,
              const double *Y, int64_t ldY, double *dYdt, int32_t precision, void *stream,
              void *workspace, int64_t workspace_bytes);

/* The CUDA source of the generated f (KIN_FEVAL_GENERATED) for a mechanism
 * description: straight-line FP64 code of Eqs. (E:mass), (E:spec-rate) and
 * (E:rxn-rate) with the mechanism's indices and constants as literals, and,
 * when the description has cp and Hf, the form with the energy equation,
 * Eq. (E:energy), whose rate constants (Eq. (E:rxn-const)) follow T. Host
 * only (no device needed). Writes at most cap - 1 characters and a NUL to buf
 * (buf may be NULL when cap is 0) and returns the full length, so a call with
 * cap 0 sizes the buffer. KIN_EINVAL for an invalid description,
 * KIN_EUNSUPPORTED beyond KIN_GEN_MAX_SPECIES / KIN_GEN_MAX_REACTIONS. */
int64_t kin_generated_f_source(const kin_mech_desc *desc, char *buf, int64_t cap);

/* Library version string. */
const char *kin_version(void);

#ifdef __cplusplus
}
#endif
#endif /* KIN_H */
