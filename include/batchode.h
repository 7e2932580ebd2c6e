/*
 * batchode.h -- C ABI of the GB300 batched ODE integration library
 * (libbatchode.so).
 *
 * Integrates very large batches of independent small ODE systems
 * dy/dt = f(t, y, g) (the paper's Eq. ode, Section 2), each with its own
 * initial state y(t0) and constant parameters g, by
 *   - rkck_integrate: adaptive fifth-order Runge-Kutta-Cash-Karp
 *     (Section 2.1: Table 1, the k1..k6 equations, the error scale and the
 *     step-size rule Eq. E:hnew; control flow of the rkckDriver listing,
 *     Section 3.1), and
 *   - rkc_integrate: stabilised second-order Runge-Kutta-Chebyshev
 *     (Section 2.2: Eqs. E:rkc0-E:rkcs, Eq. E:rmsE, Eqs. dtnp1 / rkc-f, the
 *     initial-step and stage-count rules; control flow of the rkcDriver
 *     listing, Section 3.2, and the Appendix power method).
 * The right-hand side is one of a small registry of built-in families
 * (ode_rhs_register).  No PyTorch or CUDA type appears in these signatures;
 * a stream is passed as an opaque pointer (a cudaStream_t, NULL = the legacy
 * default stream).
 *
 * Memory layout (Section 3, "structure of arrays"): unknown j of system i is
 * at y[i + nsys * j]; parameter p of system i at params[i + nsys * p].  All
 * arrays are caller-owned.  By default every array pointer is a DEVICE
 * pointer on the current device; with opts->io == ODE_IO_HOST they are host
 * pointers (pinned memory gives asynchronous copies) and the call copies
 * them in and out through a library-owned device workspace, then
 * synchronises the stream before returning.  y_out may alias y0.
 *
 * Errors: every entry point returns ODE_OK (0) on success or a negative
 * ODE_ERR_* code; ode_last_error() then describes the failure (thread-local
 * string, valid until the next call on the same thread).  Argument errors
 * are detected on the host before any launch.  Per-system outcomes are
 * written to stats->status: ODE_ST_OK, ODE_ST_H_UNDERFLOW,
 * ODE_ST_MAX_ATTEMPTS, ODE_ST_NONFINITE, optionally OR-ed with the warning
 * bit ODE_ST_SPECRAD_NOCONV (RKC power method stopped at 50 iterations).
 * Launches are asynchronous on the stream unless io == ODE_IO_HOST or
 * opts->sync != 0.
 */
#ifndef BATCHODE_H
#define BATCHODE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define ODE_OK 0
#define ODE_ERR_ARG (-1)          /* invalid argument (null, size, tolerance, interval) */
#define ODE_ERR_HANDLE (-2)       /* unknown or released rhs handle */
#define ODE_ERR_CUDA (-3)         /* a CUDA runtime call failed */
#define ODE_ERR_UNSUPPORTED (-4)  /* combination not built (e.g. dimension too large) */
#define ODE_ERR_NOMEM (-5)        /* workspace allocation failed */

/* per-system status codes */
#define ODE_ST_OK 0
#define ODE_ST_H_UNDERFLOW 1      /* step size fell below the minimum */
#define ODE_ST_MAX_ATTEMPTS 2     /* attempt cap reached before tend */
#define ODE_ST_NONFINITE 3        /* NaN error estimate or non-finite state */
#define ODE_ST_SPECRAD_NOCONV 256 /* warning bit: power method did not converge */
#define ODE_ST_PROPOSED 512       /* information bit: RKC took a proposed h0 / sigma0 or the network's bound (opts.mlp) */

/* right-hand-side families */
#define ODE_RHS_VDP 1        /* van der Pol: y1' = y2, y2' = mu (1 - y1^2) y2 - y1; params [mu]; neq 2 */
#define ODE_RHS_VDP_CHAIN 2  /* n van der Pol oscillators [x_1..x_n, v_1..v_n], diffusive position
                                coupling with free ends; params [mu]; neq 2n */
#define ODE_RHS_BRUSS1D 3    /* 1D Brusselator on n interior points [u_1..u_n, v_1..v_n], Dirichlet
                                ghosts u = ubc, v = vbc; params [a] (diffusion); neq 2n */
#define ODE_RHS_MASSACTION 4 /* mass-action kinetics (Section 4.2 omega_i with constant T), Arrhenius
                                k_j = clip(10^log10A_j T^beta_j exp(-Ea_j / T), kmin, kmax);
                                params [T]; neq = n_species */
#define ODE_RHS_KINETICS 6   /* constant-volume kinetics with a temperature equation (Section 4.2):
                                state (T, Y_1..Y_S), C_i = rho Y_i / W_i, irreversible Arrhenius
                                reactions (the mass-action fields of the descriptor, S species),
                                dY_i/dt = W_i omega_i / rho, dT/dt = -sum e_i omega_i W_i / (rho c_v)
                                with polynomial thermodynamics; params [rho]; neq = S + 1 <= 64,
                                at most 1024 reactions; RKC with the power method only */
#define ODE_RHS_NBODY 5      /* planar n-body gravity (the Pleiades problem's form, Section 4.1),
                                [x_1..x_n, y_1..y_n, u_1..u_n, v_1..v_n]: x' = u, y' = v,
                                (u_i', v_i') = G sum_{j != i} m_j d_ij / |d_ij|^3,
                                d_ij = (x_j - x_i, y_j - y_i), j ascending; masses from the
                                descriptor; params [G]; neq 4n, n <= 16 */

/* precision of the integrator */
#define ODE_PREC_FP64 0      /* plain form: every operation in FP64, as the paper's listings */
#define ODE_PREC_MIXED 1     /* FP32 RHS and stage arithmetic with Kahan-compensated FP32 state;
                                FP64 time, step size, error-norm accumulation and Chebyshev
                                coefficients */
#define ODE_PREC_MIXED_LEAN 2 /* FP32 RHS, stages, step size, spectral radius and error norms,
                                Kahan-compensated FP32 state; FP64 kept where rounding accumulates
                                -- the time t -- and for the Chebyshev coefficients.  The FP64 pipe
                                of this GPU runs at 1/64 of the FP32 rate, so every FP64 instruction
                                of the step-size bookkeeping costs as much as ~64 FP32 ones */
#define ODE_PREC_F2 3        /* RKC; RKCK for van der Pol systems and chains: state, stages
                                (RKCK: the increments k_i), evaluation points and right-hand side in
                                two-float arithmetic (each value an unevaluated sum of two FP32
                                words, ~48 significant bits, FP32 instructions only); FP64 time,
                                step size, spectral radius and error-norm accumulation; Chebyshev
                                coefficients from the FP64 table as word pairs.  Follows the FP64
                                form's step sequence, where FP32 evaluation points do not: at
                                rtol 1e-6 their rounding is several percent of the error estimate
                                of Eq. E:rmsE.  Families: van der Pol, Brusselator, mass-action
                                (RKC); van der Pol, oscillator chains (RKCK: FP64 time and step
                                size, FP32 error ratio) */
#define ODE_PREC_F2_LEAN 4   /* as ODE_PREC_F2 with FP32 step size, spectral radius and error norm
                                and the remaining interval as an FP32 pair (no FP64 instruction in
                                the step loop) */

/* how systems map onto the GPU */
#define ODE_MAP_AUTO 0       /* uniform batches: the first call with >= 32768 systems times the
                                thread and queue mappings at several block sizes on its first
                                systems (output to scratch; the host waits for these runs), and
                                the choice is cached per rhs / method / precision / device.
                                Smaller batches, and calls on a capturing stream, use
                                ODE_MAP_THREAD with 128-thread blocks.  Ragged plans: see
                                ode_ragged_plan_create */
#define ODE_MAP_THREAD 1     /* one thread per system, one launch over the batch (the paper's) */
#define ODE_MAP_QUEUE 2      /* persistent kernel, one thread per system, systems pulled from a
                                device work queue one at a time as lanes finish */

#define ODE_IO_DEVICE 0
#define ODE_IO_HOST 1

/* right-hand-side code generation (mass-action networks) */
#define ODE_CODEGEN_AUTO 0   /* compile the network into straight-line device code at first use
                                (NVRTC), falling back to the generic kernels if NVRTC is absent */
#define ODE_CODEGEN_OFF 1    /* generic kernels that read the network from kernel parameters */
#define ODE_CODEGEN_ON 2     /* generated code or ODE_ERR_UNSUPPORTED */

typedef struct {
    int32_t kind;         /* ODE_RHS_* */
    int32_t neq;          /* unknowns per system */
    int32_t n_params;     /* per-system parameters (1 for every built-in family) */
    /* ODE_RHS_MASSACTION only: R reactions, each with n_reac[j] (1 or 2)
     * reactant and n_prod[j] (1 or 2) product species (indices in
     * [0, neq), a repeated species counts twice), stored in reac[2 j + q]
     * and prod[2 j + q]; Arrhenius log10A, beta, Ea (Kelvin) per reaction
     * and the clip band [kmin, kmax].  Host pointers, copied. */
    int32_t n_reactions;
    const int32_t* n_reac;
    const int32_t* reac;
    const int32_t* n_prod;
    const int32_t* prod;
    const double* log10A;
    const double* beta;
    const double* Ea;
    double kmin, kmax;
    /* ODE_RHS_BRUSS1D only */
    double bruss_A, bruss_B, bruss_ubc, bruss_vbc;
    /* ODE_RHS_VDP_CHAIN only */
    double coupling;
    /* ODE_RHS_NBODY only: neq / 4 body masses (host pointer, copied; > 0) */
    const double* masses;
    /* ODE_RHS_KINETICS only (with the reaction fields above): molecular
     * weights [S] in kg/mol and thermodynamic coefficients [S][4]
     * (cp/R = a0 + a1 T + a2 T^2, h/(R T) = a0 + a1 T/2 + a2 T^2/3 + a3/T);
     * host pointers, copied to the device at registration */
    const double* mol_weights;
    const double* thermo;
} ode_rhs_desc;

typedef struct {
    int32_t precision;     /* ODE_PREC_* (default FP64) */
    int32_t mapping;       /* ODE_MAP_* (default AUTO) */
    int32_t max_attempts;  /* per-system attempt cap; <= 0 means 1,000,000 */
    int32_t block_size;    /* threads per block; 0 = tuned/default */
    int32_t io;            /* ODE_IO_DEVICE or ODE_IO_HOST */
    int32_t sync;          /* nonzero: synchronise the stream before returning */
    int32_t codegen;       /* ODE_CODEGEN_* (default AUTO) */
    int32_t cost_kind;     /* element type of `cost`: 0 = float32, 1 = int32 (e.g. a previous n_rhs) */
    int32_t carry_mode;    /* ODE_CARRY_CONTINUE (default) or ODE_CARRY_RESTART, see `carry` */
    int32_t specrad;       /* RKC spectral radius: ODE_SPECRAD_POWER (default) / _GERSHGORIN / _POWER_CAPPED */
    int32_t mlp;           /* proposal network handle (ode_mlp_create) evaluated in-kernel, 0 = none; see below */
    int32_t log_sr_every;  /* stride of the spectral-radius training log (<= 0: 1); see log_sr */
    int32_t log_sr_records;/* records per system in log_sr */
    int32_t reserved[3];   /* must be zero */
    /* RKC, mixed and two-float precisions: optional per-system proposals
     * [nsys] (device arrays, NaN = none) of the initial step and the
     * spectral-radius bound, e.g. from ode_mlp_propose.  A system with a
     * finite positive sigma0 skips the initial power method; with a finite
     * positive h0 beside it, the Euler trial step as well (it starts from
     * h0), otherwise the trial sets the first step as without a proposal.
     * The error test still judges every step and the first rejection hands
     * the system back to the power method (Appendix). */
    const float* h0;
    const float* sigma0;
    /* RKC, ODE_PREC_FP64: optional training log [nsys][neq + 4] (device):
     * at each system's first accepted step, log max(|y_k|, 1e-30) for every
     * component, the parameter, log h and log sigma of that step; when the
     * system finishes, log of its right-hand-side evaluations (n_rhs). */
    float* log_xy;
    /* Optional per-system cost estimates [nsys] (device, io DEVICE only;
     * float32 or, with cost_kind = 1, int32; larger = more work, e.g. the
     * previous call's n_rhs counters or the cost that ode_mlp_propose
     * predicts; NaN or <= 0 counts as cheapest).  When
     * given, the systems are taken longest-first: the library sorts them
     * into 65536 classes spread about log-uniformly over the batch's range
     * of costs, with its own kernels, and the integration kernel reads them
     * through that order.  Results do not
     * depend on the order; only the time does (lanes of a warp then hold
     * systems of similar cost, and the long ones start first).  Not in the
     * paper, whose mapping takes the systems in index order. */
    const float* cost;
    /* Optional warm-restart state, read and written (device, io DEVICE only;
     * SoA: word w of system i at carry[i + nsys * w], ODE_CARRY_WORDS(neq)
     * words per system).  The paper's outer loop (Section 3) calls the
     * integrator once per global step and every call restarts cold; it
     * notes that carrying step information across calls could help.  Words:
     * 0 valid flag (1.0 = usable), 1 time reached, 2 the controller's next
     * step size h, 3 sigma, 4 h_old, 5 err_old, 6 accepted-step count, 7 the
     * count at the last spectral-radius estimate, 8 rejected flag (RKC; RKCK
     * uses words 0-2 and writes zeros elsewhere), then the power-method
     * eigenvector v (neq words, RKC).  A system whose carry is valid resumes
     * the step-size controller and the 25-step spectral-radius schedule
     * instead of running the power method and the trial step; F(t0, y0) is
     * evaluated again.  On return every system's carry is written (valid
     * unless it ended in H_UNDERFLOW or NONFINITE); zero the array for a
     * cold start.  carry_mode ODE_CARRY_CONTINUE resumes everything: a run
     * stopped by the attempt cap and continued from the time it reached
     * repeats the uninterrupted run step for step.  ODE_CARRY_RESTART keeps
     * the controller (h, h_old, err_old) and the eigenvector but estimates
     * sigma again at the start of the call (from the carried eigenvector,
     * so in few iterations) and counts the 25-step schedule from there --
     * the choice for operator splitting, where the state changes between
     * calls, and faster in a batch: the lanes of a warp then re-estimate
     * together instead of at scattered steps.  The error test judges every
     * step either way. */
    double* carry;
    /* RKC, ODE_PREC_FP64: optional training log of the spectral-radius
     * estimates [nsys][log_sr_records][neq + 2] (device).  The power
     * method's estimates of a system are numbered q = 0, 1, ... (q = 0 at
     * the start, then the 25-step schedule and the estimates after
     * rejections, Appendix); estimate q with q % log_sr_every == 0 writes
     * record q / log_sr_every, if that is below log_sr_records:
     * log max(|y_k|, 1e-30) of the state it was taken at, the parameter
     * and log sigma (1.2 x the power method's value).  Records a system
     * never reaches are left as they were (fill the array with NaN first).
     *
     * opts.mlp (ODE_PREC_F2 / ODE_PREC_F2_LEAN, RKC): a network trained to
     * predict log sigma from those features (n_in = neq + 1), evaluated in
     * the integration kernel wherever the power method would run -- at the
     * start (unless sigma0 is given) and every 25 accepted steps, but never
     * after a rejection.  The warp evaluates it for all its systems at such
     * a point at once, on the tensor cores (BF16, FP32 accumulation).  Its
     * bound replaces the power method when it is finite, positive, at
     * least half the system's previous bound and its features lie inside
     * the network's training box widened by 5 % of its width on each side;
     * otherwise the power method runs.  Systems that took a bound from it
     * carry ODE_ST_PROPOSED.  Where a system runs on more than one thread
     * (warp or team mappings) the power method runs as without a network.
     * The network must stay alive until the integration has finished.
     * Errors: ODE_ERR_HANDLE for an unknown network, ODE_ERR_ARG for a
     * network of another input count, ODE_ERR_UNSUPPORTED for another
     * method or precision or a right-hand side without parameters. */
    float* log_sr;
} ode_opts;

#define ODE_CARRY_CONTINUE 0
#define ODE_CARRY_RESTART 1

/* RKC spectral-radius estimate (opts->specrad).  The Appendix gives the
 * nonlinear power method and names the Gershgorin circle theorem as an
 * upper-bound alternative: every eigenvalue of the Jacobian J lies in a
 * disc centred at J_ii of radius sum_{j != i} |J_ij|, so the spectral radius
 * is at most G = max_i sum_j |J_ij| (the analytic Jacobian of each built-in
 * right-hand side; row sums over the columns in increasing order).
 *   POWER         the Appendix method, 1.2 x its estimate (the paper's)
 *   GERSHGORIN    sigma = G wherever the power method would run: no
 *                 right-hand-side evaluations, an estimate never below the
 *                 true radius, but often above it (more stages per step)
 *   POWER_CAPPED  the power method's value capped at G (the bound as a
 *                 safety check: the 20 % margin never exceeds a rigorous bound) */
#define ODE_SPECRAD_POWER 0
#define ODE_SPECRAD_GERSHGORIN 1
#define ODE_SPECRAD_POWER_CAPPED 2

#define ODE_CARRY_FIXED 9
#define ODE_CARRY_WORDS(neq) ((neq) + ODE_CARRY_FIXED)

/* Per-system outputs, each an array of nsys int32 (device pointers unless
 * io == ODE_IO_HOST) or NULL when not wanted.  n_rhs counts RHS evaluations
 * as the algorithm defines them: 6 per RKCK attempt; for RKC one initial
 * F(t0), one per initial-step trial, m per m-stage attempt and one per
 * power-method iteration. */
typedef struct {
    int32_t* n_accept;
    int32_t* n_reject;
    int32_t* n_rhs;
    int32_t* n_specrad_iter;
    int32_t* status;
} ode_stats;

/* Register a right-hand side.  The descriptor (and for mass-action the
 * network arrays) is validated and copied; *rhs_handle receives a positive
 * handle.  Errors: ODE_ERR_ARG for an unknown kind, neq out of range
 * (VDP: 2; chain: even, 2..128; Brusselator: even, 2..256; mass-action: 1..32 species,
 * 1..64 reactions; n-body: multiple of 4, 4..64; kinetics: 2..64, i.e. T and
 * up to 63 species, 1..1024 reactions) or bad indices / masses / mechanism
 * data. */
int ode_rhs_register(const ode_rhs_desc* desc, int32_t* rhs_handle);

/* Release a handle.  ODE_ERR_HANDLE if it is not registered. */
int ode_rhs_release(int32_t rhs_handle);

/* Compile ahead of time the generated kernels of a registered mass-action
 * network for one method (0 = RKCK, 1 = RKC) and precision (ODE_PREC_*),
 * so that the first integrate call (or a CUDA graph capture) does not pay
 * the compilation.  Kernels are cached in memory per device and as cubins
 * on disk (directory BATCHODE_CACHE_DIR, else $HOME/.cache/batchode).
 * BATCHODE_JIT_MINBLOCKS overrides the register budget of the generated
 * kernels (that many 128-thread blocks resident per SM; defaults 2 for
 * ODE_PREC_FP64, 3 for the mixed forms), BATCHODE_JIT_LOCKSTEP (0-2) the
 * one-launch kernel's step-end hold (2, block-wide, for the two-float forms;
 * 0, warp-level, for the others) and BATCHODE_JIT_VERBOSE=1 prints the
 * compiler's resource report to stderr.
 * Without a visible device only the compilation (and disk cache) happens.
 * Other families need no preparation and return ODE_OK.  Errors:
 * ODE_ERR_HANDLE, ODE_ERR_ARG, ODE_ERR_UNSUPPORTED (NVRTC missing or the
 * compilation failed; ode_last_error has the log), ODE_ERR_CUDA. */
int ode_rhs_prepare(int32_t rhs_handle, int32_t method, int32_t precision);

/* Integrate nsys systems from t0 to tend with the adaptive RKCK method.
 * y0, params: [neq][nsys] and [n_params][nsys] FP64; y_out: [neq][nsys].
 * rtol > 0, atol >= 0, tend > t0 (tend == t0 copies y0).  opts may be NULL
 * (defaults).  Precision forms: FP64 and the FP32 forms for every family;
 * the two-float forms for van der Pol systems and oscillator chains (other
 * families: ODE_ERR_UNSUPPORTED before any device work).  Errors:
 * ODE_ERR_ARG, ODE_ERR_HANDLE, ODE_ERR_CUDA, ODE_ERR_NOMEM,
 * ODE_ERR_UNSUPPORTED. */
int rkck_integrate(int32_t rhs, int64_t nsys, const double* y0, const double* params, double t0,
                   double tend, double rtol, double atol, const ode_opts* opts, double* y_out,
                   const ode_stats* stats, void* stream);

/* Same contract with the adaptive RKC method (spectral radius by the
 * nonlinear power method, re-estimated every 25 accepted steps and after a
 * rejection). */
int rkc_integrate(int32_t rhs, int64_t nsys, const double* y0, const double* params, double t0,
                  double tend, double rtol, double atol, const ode_opts* opts, double* y_out,
                  const ode_stats* stats, void* stream);

/* RKC integration for callers that cannot allocate GPU memory.
 *
 * Some callers may not call cudaMalloc at all: code running inside another
 * framework's memory pool or a fixed memory budget, hosts that forbid
 * growing the device footprint after start-up, or code that must not fail
 * on an allocation halfway through a job.  rkc_integrate allocates a
 * workspace on first use (and grows a staging buffer for host arrays);
 * this entry point allocates nothing.  Its scratch -- the work-queue
 * cursor, an RKC coefficient table for stage counts up to 32 and the
 * staging area for the caller's arrays -- lives in one statically sized
 * device array of ODE_NOALLOC_SCRATCH_BYTES (16 MiB) that every GPU which
 * loads this library holds until the process exits.  The paper has no
 * counterpart; it is a packaging of the same integrator.
 *
 * Same arguments and results as rkc_integrate (every built-in family;
 * opts->specrad as there, kinetics with the power method only), except: y0,
 * params, y_out and the stats arrays are HOST pointers (pinned memory gives
 * asynchronous copies; y_out may alias y0); precisions ODE_PREC_FP64,
 * ODE_PREC_MIXED and ODE_PREC_MIXED_LEAN only (others: ODE_ERR_ARG);
 * opts->mapping ODE_MAP_THREAD runs one launch over the batch and any other
 * value the persistent queue (no tuning runs: they would need scratch
 * output); opts->io and opts->codegen are ignored (the built-in kernels
 * are used, never run-time generated ones, since loading generated code
 * allocates), and so are opts->h0, sigma0, log_xy, cost, carry and
 * carry_mode; opts->mlp and log_sr are rejected (ODE_ERR_ARG).  A batch whose staged arrays need more than the
 * scratch offers -- nsys * 8 * (neq + n_params) bytes plus 4 * nsys per
 * requested counter array, each rounded up to 256 bytes, against 16 MiB
 * minus the cursor and table -- is rejected with ODE_ERR_ARG before any GPU
 * work; split such a batch into several calls.
 *
 * The first call on each device does the set-up (looks up the array's
 * device address with the device current and builds the coefficient table
 * into it, then synchronises), so make that first call before any stream
 * capture.  Every call shares the array and finds the previous call's
 * contents there: the cursor is cleared on every call, and every staged or
 * output element is rewritten.  Calls that overlapped on the GPU would race
 * on the array; this entry point serialises its own calls with a process-wide
 * lock and synchronises the stream before returning -- on error returns too,
 * once anything was queued. */
#define ODE_NOALLOC_SCRATCH_BYTES 16777216 /* 16 MiB */
int rkc_integrate_noalloc(int32_t rhs, int64_t nsys, const double* y0, const double* params, double t0,
                          double tend, double rtol, double atol, const ode_opts* opts, double* y_out,
                          const ode_stats* stats, void* stream);

/* ---------------------------------------------------------------------
 * Ragged batches: systems of different sizes, families and methods in one
 * call (independent systems, Section 2, Eq. ode).  A plan buckets the
 * systems by family, method and size class (8, 16, 32, 64, 128, 256
 * unknowns), orders each bucket largest-first, chooses each bucket's kernel
 * shape (lanes per system, grid points per lane, block size) and captures all
 * buckets' persistent-queue kernels, on parallel branches, in one CUDA graph;
 * ode_ragged_plan_launch replays it (in place when y_out == y0, so a plan can
 * integrate the same buffers again and again).  opts->mapping: ODE_MAP_AUTO
 * times the candidate shapes, block sizes and mappings (queue or one launch)
 * on a sample of each bucket (results cached per family / method /
 * precision / size class; an in-place plan's sample writes to a temporary
 * copy of the state), ODE_MAP_THREAD is the paper's
 * one-thread-per-system mapping with 64-thread blocks, ODE_MAP_QUEUE the
 * default warp-per-system shape; opts->h0, sigma0, log_xy, cost and carry
 * are ignored (a plan orders each bucket by system size).  Families: Brusselator and oscillator
 * chains (register each family once with its largest neq).  Layout: system
 * i's components are contiguous from offset[i].  opts->precision: any form;
 * with a two-float form (ODE_PREC_F2, ODE_PREC_F2_LEAN) the buckets take the
 * two-float kernels (warp-wide teams: Brusselator grids by RKC, oscillator
 * chains by RKCK or RKC) and Brusselator grids by RKCK, for which no
 * two-float form is built, the FP64 kernels, so that every system of the
 * plan keeps FP64-class accuracy. */
typedef struct {
    int64_t nsys;
    const int32_t* rhs;     /* HOST [nsys]: registered handle of each system's family */
    const int32_t* method;  /* HOST [nsys]: 0 = RKCK, 1 = RKC */
    const int32_t* neq;     /* HOST [nsys]: unknowns of each system (even, <= the handle's neq) */
    const int64_t* offset;  /* HOST [nsys]: start of each system in y0 / y_out */
    const double* y0;       /* DEVICE [sum neq] */
    const double* params;   /* DEVICE [nsys]: one parameter per system */
    const double* t0;       /* DEVICE [nsys] */
    const double* tend;     /* DEVICE [nsys] */
    const double* rtol;     /* DEVICE [nsys] */
    const double* atol;     /* DEVICE [nsys] */
} ode_ragged_batch;

/* Builds a plan (tuning runs real integrations of samples on `stream`, then
 * the graph is captured); *plan receives its handle.  Arrays and y_out /
 * stats (device, indexed by system) must stay valid while the plan is used.
 * Errors: ODE_ERR_ARG, ODE_ERR_HANDLE, ODE_ERR_UNSUPPORTED, ODE_ERR_NOMEM,
 * ODE_ERR_CUDA. */
int ode_ragged_plan_create(const ode_ragged_batch* batch, const ode_opts* opts, double* y_out,
                           const ode_stats* stats, void* stream, int64_t* plan);
/* Integrates the whole batch once (asynchronous on stream). */
int ode_ragged_plan_launch(int64_t plan, void* stream);
/* Bucket descriptions: 8 int32 per bucket (family, method, size class,
 * systems, lanes per system, grid points per lane (0 = by size), block size,
 * mapping), up to `capacity` buckets; *n_buckets gets the count. */
int ode_ragged_plan_info(int64_t plan, int32_t* n_buckets, int32_t* desc, int32_t capacity);
int ode_ragged_plan_destroy(int64_t plan);

/* ---------------------------------------------------------------------
 * Learned initial step / spectral-radius / cost proposal.  Not in the
 * paper: the paper starts every RKC system with a power-method estimate
 * (Appendix) and an Euler trial step (Section 2.2) and takes the systems in
 * index order; this network proposes the first two from the initial state
 * and predicts each system's cost, which orders the batch (ode_opts.cost).
 * MLP n_in -> 64 -> 64 -> 3 with SiLU, FP32 master weights used as BF16
 * with FP32 accumulation (CUDA cores), inputs log max(|y_k|, 1e-30) for
 * each component plus the parameter (normalised by statistics of the
 * training set), outputs log h0, log sigma and log cost (right-hand-side
 * evaluations of the whole integration).  Training minimises squared error
 * on log h0 and log cost plus a pinball loss (quantile 0.9) on log sigma,
 * so sigma leans to over-estimates, with Adam.  A NaN target is no
 * target: it adds nothing to the loss, its gradient or the target's
 * normalisation (so records of the spectral-radius log, which have a sigma
 * target only, train beside the first-step records).  Device arrays
 * throughout, rows contiguous (X [n][n_in], Y [n][3]); returns ODE_OK or
 * ODE_ERR_*.
 * The parameter vector layout: W1 [64][n_in], b1 [64], W2 [64][64],
 * b2 [64], W3 [3][64], b3 [3]; the normalisation block: x_mean, x_scale,
 * x_min, x_max [ODE_MLP_MAX_IN each], y_mean, y_scale [3 each]. */
#define ODE_MLP_HIDDEN 64
#define ODE_MLP_MAX_IN 33
#define ODE_MLP_OUT 3
#define ODE_MLP_NORM_FLOATS 138

typedef struct {
    int32_t epochs;   /* passes over the data */
    int32_t batch;    /* rows per Adam step */
    float lr;         /* Adam learning rate */
    int32_t pad;      /* must be zero */
    uint64_t seed;    /* shuffling seed */
} ode_train_opts;

int ode_mlp_create(int32_t n_in, uint64_t seed, int32_t* mlp_handle);   /* Glorot-uniform init */
int ode_mlp_release(int32_t mlp_handle);
int ode_mlp_num_params(int32_t n_in);                                     /* -1 if n_in is out of range */
/* mean / standard deviation / range of every input and target column */
int ode_mlp_fit_normalization(int32_t mlp_handle, const float* X, const float* Y, int64_t n, void* stream);
/* epochs of shuffled minibatch Adam; loss_history (host, [epochs]) gets each epoch's mean loss */
int ode_mlp_train(int32_t mlp_handle, const float* X, const float* Y, int64_t n, const ode_train_opts* opts,
                  float* loss_history, void* stream);
/* gradient of the mean loss over the n rows w.r.t. the parameters (device grad_out [num_params]);
 * *loss_out (host) = the mean loss; synchronous */
int ode_mlp_gradient(int32_t mlp_handle, const float* X, const float* Y, int64_t n, float* grad_out,
                     float* loss_out, void* stream);
/* outputs (log h0, log sigma, log cost) for raw feature rows: out [n][3] */
int ode_mlp_apply(int32_t mlp_handle, const float* X, int64_t n, float* out, void* stream);
/* proposals for an SoA batch (y0 [neq][nsys], params [1][nsys], FP64): h0 and sigma0 [nsys], NaN where
 * an input lies outside the training range widened by `margin` of its width, or an output is not finite;
 * cost [nsys] (may be NULL): the predicted right-hand-side evaluations, NaN only where not finite */
int ode_mlp_propose(int32_t mlp_handle, int64_t nsys, int32_t neq, const double* y0, const double* params,
                    float margin, float* h0, float* sigma0, float* cost, void* stream);
/* outputs 0 and 1 (log h0, log sigma) for raw feature rows X [n][n_in], evaluated as the integration
 * kernels evaluate the network in-kernel (opts.mlp): one warp per 32 rows, mma.sync products with BF16
 * inputs, weights and activations and FP32 accumulation; out [n][2]; no box check */
int ode_mlp_apply_warp(int32_t mlp_handle, const float* X, int64_t n, float* out, void* stream);
/* host copies of the FP32 parameters [num_params] and the normalisation block (either may be NULL) */
int ode_mlp_get_params(int32_t mlp_handle, float* params, float* norm);
int ode_mlp_set_params(int32_t mlp_handle, const float* params, const float* norm);

/* The mapping and block size an ODE_MAP_AUTO call with these options
 * (method 0 = RKCK, 1 = RKC; precision, codegen and block_size as in
 * ode_opts) uses on the current device.  Returns ODE_OK when they come from
 * a timing already made, ODE_ERR_UNSUPPORTED (outputs still set) when the
 * untuned default would be used, ODE_ERR_HANDLE / ODE_ERR_ARG otherwise. */
int ode_mapping_info(int32_t rhs_handle, int32_t method, int32_t precision, int32_t codegen, int32_t block_size,
                     int32_t* mapping, int32_t* block);

/* The longest-first order that opts->cost gives a batch, on its own:
 * index [n] (device int32) receives the permutation of 0..n-1 whose cost
 * classes do not increase.  With lo and hi the smallest and largest bit
 * pattern (as uint32) of the positive costs, a positive cost c is in class
 * 1 + (bits(c) - lo) * 65535 / (hi - lo + 1) (integer division; positive
 * floats order like their bit patterns, which grow about like log2 c), and
 * NaN and values <= 0 are in class 0.  Systems of one class appear in an
 * unspecified order.  cost: device [n].  Asynchronous on `stream`;
 * n <= 2^31 - 1.  No counterpart in the paper. */
int ode_cost_order(const float* cost, int64_t n, int32_t* index, void* stream);
/* The same for int32 costs (e.g. n_rhs counters), each taken as a float. */
int ode_cost_order_i32(const int32_t* cost, int64_t n, int32_t* index, void* stream);

/* Forget every cached ODE_MAP_AUTO timing (uniform calls and ragged plans),
 * so that the next such call or plan times its candidates again (after a
 * change of the generated kernels' occupancy setting, say).  No counterpart
 * in the paper, whose mapping is fixed.  Existing plans keep their shapes.
 * Always returns ODE_OK. */
int ode_tuning_reset(void);

/* Description of the last error on this thread ("" if none). */
const char* ode_last_error(void);

/* Library version string. */
const char* ode_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BATCHODE_H */
