/*
 * rfb_soc.h - C ABI of the GB300 steady state-of-charge solver.
 *
 * The library computes the steady state of the state-of-charge PDE of Emanuel & Rycroft,
 * "Digital Twin for Porous Electrodes in Redox Flow Batteries" (arXiv 2502.08034),
 * Eq. nernst-planck-soc (Sec. II.D):
 *     ds/dt = -u . grad s + D lap s + k0 a R~(s),
 * with the affine rate law R~(s) = e^{alpha V~} (1 - (1 + e^{-V~}) s)
 * (Eq. rate-from-soc-gen), V~ = n_e V_ar / V_T (Eq. Vart-def), by explicit pseudo-time
 * stepping on a voxel lattice (the explicit reformulation of Sec. III.C), plus the
 * mass-transport utilisation U_mt (Eq. umt-def, Algorithm 7).
 *
 * Discretisation (identical in every entry point):
 *   - lattice nx * ny * nz, cell size dx; flow enters through the low-z face of plane
 *     k = 0 (inlet) and leaves through the high-z face of plane k = nz-1 (outlet);
 *     cell index c = i + nx*(j + ny*k);
 *   - first-order upwind advection by the given face velocities (times the velocity
 *     scale beta), 7-point diffusion between fluid cells, no flux through side walls and
 *     fiber faces, inlet value s_in imposed on the inlet face (diffusive term
 *     (2D/dx^2)(s_in - s_c); RFB_INLET_GHOST gives (D/dx^2)(s_in - s_c)), zero-gradient
 *     outlet;
 *   - reaction k0 a_c R~(s_c) with a_c = m_c n_wall(c) / dx, n_wall = number of fiber
 *     6-neighbours (the voxel form of the cut-cell specific area a = A/V, Sec. III.B),
 *     m_c an optional per-cell area multiplier (default 1);
 *   - "overpotential" eta [V] is the activation overpotential at s = 1/2 with
 *     phi_L = 0 (Eq. etat-from-s), i.e. V_ar = -eta; eta < 0 is reducing.
 *   - residual r = tau * RMS over unknown cells of RHS(s) = (tau/dt) ||ds||_RMS
 *     (Eq. convergence-bv-change), tau = V_fluid / Q, Q = beta * sum_inlet W dx^2.
 *
 * Conventions: every call returns rfb_status; nothing throws across the ABI. A handle
 * is not thread-safe; distinct handles are independent. All work is queued on the
 * handle's CUDA stream (rfb_soc_set_stream); calls that return host values synchronise
 * that stream. Pointers marked "host or device" are interpreted per the rfb_mem_kind
 * argument; device pointers must be on the handle's device.
 */
#ifndef RFB_SOC_H
#define RFB_SOC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum rfb_status {
    RFB_OK = 0,
    RFB_ERR_INVALID_ARG = 1,   /* bad size, value, pointer or option; nothing changed */
    RFB_ERR_CUDA = 2,          /* a CUDA call failed; see rfb_soc_last_error */
    RFB_ERR_OOM = 3,           /* device allocation failed */
    RFB_ERR_NOT_CONVERGED = 4, /* max_sweeps reached; the state is valid and readable */
    RFB_ERR_NONFINITE = 5,     /* a non-finite value appeared in the state or residual */
    RFB_ERR_STATE = 6,         /* call needs a state that is not there (e.g. no solve) */
    RFB_ERR_UNSUPPORTED = 7    /* option not built into this library */
} rfb_status;

typedef enum rfb_mem_kind { RFB_MEM_HOST = 0, RFB_MEM_DEVICE = 1 } rfb_mem_kind;

typedef enum rfb_precision {
    RFB_PREC_FP64 = 0,   /* FP64 sweeps and reductions */
    RFB_PREC_MIXED = 1   /* FP32 correction sweeps; defects in double-float arithmetic
                            (FP32 pairs, ~48 bits) with FP64 reductions, switching to FP64
                            defects near that arithmetic's floor; FP64 state and a final
                            FP64 check that gives the returned residual and outputs */
} rfb_precision;

typedef enum rfb_inlet_bc { RFB_INLET_FACE = 0, RFB_INLET_GHOST = 1 } rfb_inlet_bc;

typedef enum rfb_dt_mode {
    RFB_DT_GLOBAL = 0,   /* dt = cfl / max_c d_c, d_c the diagonal of -L */
    RFB_DT_LOCAL = 1     /* dt_c = cfl / d_c per cell (same fixed point, fewer sweeps) */
} rfb_dt_mode;

/* How the overpotential argument of a solve enters the source term. With
 * eta~ = -n_e eta / V_T (Eq. etat-def; the same number as V~ = n_e V_ar / V_T with
 * V_ar = -eta):
 *   RFB_KIN_AFFINE       eta is the activation overpotential at s = 1/2 (phi_L = 0), so the
 *                        applied voltage is uniform and the rate is the affine law
 *                        R~(s) = e^{alpha V~} (1 - (1 + e^{-V~}) s) (Eq. rate-from-soc-gen);
 *                        the steady problem is linear. Default.
 *   RFB_KIN_UNIFORM_ETA  eta is the activation overpotential itself, uniform over the
 *                        electrode: R~(s) = s^alpha (1-s)^(1-alpha) (e^{alpha eta~} -
 *                        e^{(alpha-1) eta~}) (Eq. source-term-bv-gen), nonlinear in s.
 *                        FP64 precision only (solve / step return RFB_ERR_INVALID_ARG for
 *                        RFB_PREC_MIXED; batches refuse such handles). The explicit update
 *                        is clipped into [0, 1] (a guard; it does not bind at a steady
 *                        state), and the pseudo-time step is the affine law's at the same
 *                        eta. With s_in = 0 the rate vanishes everywhere at the start and
 *                        s = 0 is the (trivial) steady state. */
typedef enum rfb_kinetics_mode {
    RFB_KIN_AFFINE = 0,
    RFB_KIN_UNIFORM_ETA = 1
} rfb_kinetics_mode;

/* Butler-Volmer kinetics (Sec. II.B, parameter table). */
typedef struct rfb_kinetics {
    double k0;      /* rate constant [m/s] */
    double alpha;   /* charge-transfer coefficient, 0 < alpha < 1 */
    int32_t n_e;    /* electrons per reaction (2 for AQDS) */
    int32_t mode;   /* rfb_kinetics_mode (0 = RFB_KIN_AFFINE) */
    double T;       /* temperature [K] */
    double c0;      /* total concentration of redox species C_T [mol/m^3] */
} rfb_kinetics;

typedef struct rfb_solve_opts {
    int32_t precision;      /* rfb_precision (default RFB_PREC_FP64) */
    int32_t inlet_bc;       /* rfb_inlet_bc (default RFB_INLET_FACE) */
    int32_t dt_mode;        /* rfb_dt_mode (default RFB_DT_LOCAL) */
    int32_t check_every;    /* sweeps between FP64 residual checks (0 = automatic) */
    double cfl;             /* C_CFL in (0, 1] (default 0.4) */
    double velocity_scale;  /* beta >= 0: every face velocity is multiplied by it (1) */
    int64_t max_sweeps;     /* give up after this many sweeps (0 = 50,000,000) */
    int32_t fp32_kernel;    /* RFB_PREC_MIXED only: 0 = chosen by timing the kernels on
                               the lattice (once per lattice shape, dt mode
                               and device in a process), 1 = one sweep per launch,
                               2 = several sweeps per pass (TMA-staged, temporally
                               blocked; local steps: nx % 4 == 0; global step: nx % 16
                               == 0 and no area multiplier), the pass variant chosen by
                               timing; 3 = two-sweep passes in a persistent launch (one
                               CTA per SM, equal shares); 4 = two-sweep passes, one
                               (tile, z chunk) item per CTA; local steps only: 5 / 6 = as
                               3 / 4 with four TMA stages instead of three; 7 / 8 =
                               three-sweep passes (128 x 10 tiles, the update
                               coefficients of the two older levels in tensor memory),
                               persistent / chunked; 9 / 10 = as 7 / 8 with five delta
                               stages instead of four. Every pass is bitwise the same
                               number of one-sweep launches; check intervals are whole
                               passes */
    int32_t timeout_ms;     /* > 0: stop after the first FP64 check at or past this much
                               wall time since the call began and return
                               RFB_ERR_NOT_CONVERGED (the state is valid); 0 = none */
    int32_t reserved[6];    /* must be zero */
} rfb_solve_opts;

typedef struct rfb_solve_result {
    int64_t sweeps;          /* explicit sweeps applied by this call */
    int64_t checks;          /* FP64 residual evaluations */
    double residual;         /* tau * RMS(RHS) at the returned state */
    double I_tot;            /* total current [A], Eq. I-tot-def */
    double F_in;             /* inlet electron flow [A], advective + diffusive */
    double F_out;            /* outlet electron flow [A], Eq. electron-flow */
    double F_in_adv;         /* advective part of F_in (the paper's F_in) */
    double mass_balance_rel; /* |I_tot - (F_out - F_in)| / |I_tot|, Eq. convergence-bv-flow */
    double U;                /* utilisation I_tot / (n_e F c0 Q (1 - s_in)), Eq. utilization-def */
    double outlet_mean;      /* sum_out W s / sum_out W */
    double dt;               /* global pseudo-time step [s] (RFB_DT_LOCAL: the minimum) */
    double tau;              /* V_fluid / Q [s] */
    double time_ms;          /* wall time of the call */
    int64_t nonfinite;       /* non-finite RHS values seen at the last check */
    double sweep_ms;         /* device time of the sweep kernels (CUDA events on the
                                handle's stream around each batch of sweeps) */
    double check_ms;         /* device time of the FP64 checks (kernel + reduction) */
} rfb_solve_result;

typedef struct rfb_soc_handle rfb_soc_handle;

/* Fill opts with the defaults listed above. */
void rfb_solve_opts_default(rfb_solve_opts* opts);

/* Static string for a status code (never NULL). */
const char* rfb_status_string(rfb_status st);

/* Last error detail recorded on the handle (empty string if none; never NULL). */
const char* rfb_soc_last_error(const rfb_soc_handle* h);

/*
 * Create a solver for one lattice (Sec. III.C: the explicit operators are built once
 * per geometry and flow field).
 *   dims          nx, ny, nz >= 1 (nz >= 2)
 *   dx            cell size [m] > 0
 *   fiber_mask    N bytes, 1 = fiber (solid), 0 = fluid; layout c = i + nx*(j + ny*k)
 *   U, V, W       face velocities [m/s]: U (nx+1)*ny*nz with U[i + (nx+1)*(j + ny*k)] on
 *                 the face between cells i-1 and i; V nx*(ny+1)*nz; W nx*ny*(nz+1) with
 *                 plane 0 = inlet faces, plane nz = outlet faces. Must be finite, zero on
 *                 side walls and on every face touching a fiber cell; inlet and outlet
 *                 W must be >= 0.
 *   D             diffusivity [m^2/s] > 0
 *   kin           kinetics (k0 >= 0, 0 < alpha < 1, n_e >= 1, T > 0, c0 > 0)
 *   area_mult     nullable; N doubles > 0 (the per-cell multiplier m_c)
 *   kind          whether the array pointers are host or device memory
 *   cuda_stream   cudaStream_t to queue work on (NULL = legacy default stream)
 *   out           receives the handle
 * The library copies every input into device memory it owns; the caller may free its
 * arrays on return. Invalid inputs return RFB_ERR_INVALID_ARG with a message on *out
 * left NULL (read it with rfb_soc_last_error(NULL)).
 */
rfb_status rfb_soc_create(const int32_t dims[3], double dx, const uint8_t* fiber_mask,
                          const double* U, const double* V, const double* W, double D,
                          const rfb_kinetics* kin, const double* area_mult,
                          rfb_mem_kind kind, void* cuda_stream, rfb_soc_handle** out);

/* Release every resource of the handle. NULL-safe. */
rfb_status rfb_soc_destroy(rfb_soc_handle* h);

/* Queue subsequent work of the handle on this cudaStream_t (NULL = default stream). */
rfb_status rfb_soc_set_stream(rfb_soc_handle* h, void* cuda_stream);

/*
 * Drive the state to residual <= tol by explicit pseudo-time sweeps
 * s <- s + dt RHS(s) (Eq. nernst-planck-soc stepped to dt-independent steady state).
 *   s_in   inlet state of charge, 0 <= s_in <= 1
 *   eta    overpotential [V] (see above)
 *   tol    residual tolerance > 0
 *   opts   nullable (defaults)
 *   res    nullable; filled on return (also on NOT_CONVERGED / NONFINITE)
 * Starts from the current state if one is set (previous solve, rfb_soc_set_state or
 * rfb_soc_upsample), otherwise from s = s_in on every fluid cell.
 * RFB_PREC_MIXED: cycles of opts.check_every (default 200) FP32 correction sweeps
 * delta <- delta + dt (L delta + r) followed by a defect check that adds delta to the
 * state and refreshes r; res->residual and the outputs come from an FP64 check of the
 * returned state. Kinetics mode 1 requires RFB_PREC_FP64.
 * Returns RFB_OK, RFB_ERR_NOT_CONVERGED (state valid) or RFB_ERR_NONFINITE.
 */
rfb_status rfb_soc_solve(rfb_soc_handle* h, double s_in, double eta, double tol,
                         const rfb_solve_opts* opts, rfb_solve_result* res);

/*
 * Apply exactly n_sweeps explicit sweeps to the current state (FP64 or, with
 * RFB_PREC_MIXED, FP32 sweeps on a correction that is added to the FP64 state), then
 * evaluate the outputs into res (nullable). Starts from s = s_in if no state is set.
 */
rfb_status rfb_soc_step(rfb_soc_handle* h, double s_in, double eta, int64_t n_sweeps,
                        const rfb_solve_opts* opts, rfb_solve_result* res);

/*
 * Evaluate residual, I_tot, F_in, F_out, mass balance and U (Sec. II.C) in FP64 on the
 * current state at the operating point of the last solve/step. RFB_ERR_STATE if none.
 */
rfb_status rfb_soc_current(rfb_soc_handle* h, rfb_solve_result* res);

/*
 * Same outputs as rfb_soc_current, computed in FP64 by the matrix-free check kernel
 * (coefficients built from the face velocities; rfb_soc_current applies the assembled
 * operator, so the two agree up to rounding, ~1e-16 of the largest RHS term per cell)
 * and the same fixed-order reduction, but without touching any device memory that
 * needs allocating: the
 * per-block partial sums go to a static device array of 65,600 bytes (8192 blocks x 8
 * sums + 8 totals) that every GPU loading this library holds until the process exits.
 * The paper has no counterpart; this exists for callers that cannot allocate at the
 * moment they need the outputs, e.g. a runtime whose caching allocator owns the
 * device's memory, or a monitor on a latency-critical path that must not pay for the
 * device-wide synchronisation of cudaMalloc/cudaFree.
 *   res   host struct, filled like rfb_soc_current (sweeps = 0, checks = 1)
 * Errors: RFB_ERR_STATE without a state; RFB_ERR_INVALID_ARG if the lattice needs more
 * than 8192 reduction blocks (about nx*ny > 2,000,000; use rfb_soc_current then).
 * Every call made outside a stream capture looks up the array's device address
 * (cudaGetSymbolAddress with the handle's device current; after a cudaDeviceReset the
 * module is reloaded and the address may change). A call during a capture uses the
 * address of the last uncaptured call on that device, so make the first call on a
 * device before any stream capture begins (RFB_ERR_STATE otherwise).
 * All calls in the process share the one array and its contents stay behind after a
 * call; calls whose work overlaps on the GPU (other streams, other handles, other host
 * threads) race on it and must be serialised by the caller.
 */
rfb_status rfb_soc_current_noalloc(rfb_soc_handle* h, rfb_solve_result* res);

/*
 * Mass-transport utilisation U_mt (Eq. umt-def): the steady state of advection and
 * diffusion with s = 0 at the inlet and every fluid cell that touches a fiber held at 1
 * (Eqs. np-fast-interior/np-fast-boundary, Algorithm 7), then sum_out W s / sum_out W.
 * Independent of the kinetics and of s_in. Uses its own state buffer (the SOC state is
 * untouched). opts nullable; res (nullable) receives sweeps and residual.
 */
rfb_status rfb_soc_umt(rfb_soc_handle* h, double tol, const rfb_solve_opts* opts,
                       double* umt, rfb_solve_result* res);

/*
 * Iterative upsampling (Sec. III.A; the paper solves coarse to
 * steady state and initialises the refined problem from it by coarse-to-fine
 * interpolation). Sets fine's state to the 2x prolongation of coarse's state:
 * injection s_f(i,j,k) = s_c(i/2, j/2, k/2) for fine fluid cells with a fluid parent
 * (the coarse-to-fine comparison rule of Sec. IV); a fine fluid cell whose parent is
 * solid takes the mean of the parent's fluid 6-neighbours, else the coarse handle's
 * last s_in. The next rfb_soc_solve on fine warm-starts from it; the fixed point does
 * not depend on the start. Requires fine dims = 2 x coarse dims, fine dx = coarse dx / 2,
 * both handles on one device, and a coarse state (RFB_ERR_STATE otherwise). Synchronises
 * both handles' streams.
 */
rfb_status rfb_soc_upsample(const rfb_soc_handle* coarse, rfb_soc_handle* fine);

/*
 * Replace the per-cell reactive-area multiplier m_c (N doubles > 0, host or device;
 * NULL = all ones). The state is kept as a warm start for the next solve.
 */
rfb_status rfb_soc_set_area_mult(rfb_soc_handle* h, const double* m, rfb_mem_kind kind);

typedef enum rfb_objective {
    RFB_OBJ_I_TOT = 0,   /* total current I_tot [A], Eq. I-tot-def */
    RFB_OBJ_U = 1,       /* utilisation U, Eq. utilization-def (first form) */
    RFB_OBJ_U_MT = 2     /* mass-transport utilisation U_mt, Eq. umt-def */
} rfb_objective;

/*
 * Discrete adjoint of the steady state. The steady state solves RHS(s) = L s + b = 0
 * (linear in s by Eq. rate-from-soc-gen), so for an objective J the adjoint lam solves
 * L^T lam = -dJ/ds (transposed explicit sweeps, the downwind gather of the upwind
 * operator, same pseudo-time steps as the forward solve, to ||L^T lam + dJ/ds|| /
 * ||dJ/ds|| <= tol), and
 *   dJ/dm_c  = dJ/dm_c|explicit + lam_c k0 n_wall(c)/dx R~(s_c)
 *   dJ/dbeta = dJ/dbeta|explicit + lam . (advective part of RHS(s)) / beta.
 * I_TOT and U need a converged rfb_soc_solve at the current operating point (and area
 * multipliers); U_MT needs a converged rfb_soc_umt. dU_mt/dm is identically zero (the
 * U_mt problem has no kinetics) and is returned as zeros. velocity_scale must be > 0.
 * RFB_KIN_UNIFORM_ETA: the source is nonlinear; L above is the Jacobian dRHS/ds at the
 * converged state (transport plus k0 a_c dR~/ds on the diagonal) and R~ the mode's rate.
 *   opts             nullable; dt_mode / cfl / check_every / max_sweeps / timeout_ms are
 *                    used, and precision: RFB_PREC_FP64 (FP64 transposed sweeps) or
 *                    RFB_PREC_MIXED (FP32 sweeps of the transposed operator correcting lam,
 *                    defects g + L^T lam in double-float arithmetic, the last one confirmed
 *                    in FP64; kinetics mode 0 or U_MT, nx % 4 == 0, else
 *                    RFB_ERR_INVALID_ARG)
 *   d_area_mult      nullable; N doubles (host or device per kind) receiving dJ/dm_c
 *                    (zero on solid cells and cells without fiber neighbours)
 *   d_velocity_scale nullable; host double receiving dJ/dbeta
 *   res              nullable; sweeps, checks, residual (relative adjoint residual), and
 *                    the objective's forward values I_tot / U / outlet_mean
 */
rfb_status rfb_soc_adjoint(rfb_soc_handle* h, rfb_objective obj, double tol,
                           const rfb_solve_opts* opts, double* d_area_mult,
                           double* d_velocity_scale, rfb_mem_kind kind,
                           rfb_solve_result* res);

/* Forget the current state: the next solve/step starts from s = s_in (cold start). */
rfb_status rfb_soc_reset_state(rfb_soc_handle* h);

/* Copy the FP64 state (N doubles, solid cells 0) out to host or device memory. */
rfb_status rfb_soc_get_state(rfb_soc_handle* h, double* s, rfb_mem_kind kind);

/* Set the FP64 state (N doubles; solid-cell values are ignored). Must be finite. */
rfb_status rfb_soc_set_state(rfb_soc_handle* h, const double* s, rfb_mem_kind kind);

/*
 * Batches: many lattices of uneven size and operating points (the paper's design
 * question, how utilisation varies with geometry, flow rate and voltage, Sec. V)
 * advanced together. Each sweep over all lattices is one persistent launch whose
 * resident blocks walk a list of work items (128 x 8 column tiles times a chunk of z
 * planes, from every lattice); one correction cycle (zeroing, sweeps, fused FP64 check
 * of every lattice, convergence bookkeeping) is captured once as a CUDA graph and
 * replayed until every lattice has converged; converged lattices drop out of the work
 * list on the device. Mixed precision only (FP32 correction sweeps, FP64 checks and
 * state). The z-chunk of the work items and the sweeps per cycle are picked by a
 * built-in autotuner on the first solve (timed with CUDA events).
 */
typedef struct rfb_batch rfb_batch;

typedef struct rfb_batch_info {
    int32_t kchunk;            /* z planes per work item of the one-sweep kernel
                                  (autotuned) */
    int32_t sweeps_per_cycle;  /* sweeps between FP64 checks (autotuned or opts) */
    int32_t n_items;           /* work items over all lattices */
    int32_t grid_blocks;       /* resident blocks of the persistent launch */
    double sweep_ms;           /* autotuner: device time of one sweep of the batch */
    double check_ms;           /* autotuner: device time of one FP64 check of the batch */
    int64_t cycles;            /* correction cycles of this solve */
    double time_ms;            /* wall time of this solve */
    int64_t launches;          /* kernels launched by this batch so far */
    int64_t graph_launches;    /* graph launches of this solve, each followed by one host
                                  wait: without opts.timeout_ms a launch runs up to 64
                                  cycles in a device-driven loop (a conditional while node
                                  whose condition a kernel sets once every lattice has
                                  converged); with a timeout, one cycle per launch */
    int32_t pass_stages;       /* 0: the one-sweep kernel ran; 3 / 4: the batched two-sweep
                                  pass with that many TMA stages */
    int32_t pass_chunk;        /* z planes per work item of the two-sweep pass */
    int32_t pass_tile_cols;    /* interior columns of a tile of the two-sweep pass: 128 (one
                                  CTA per SM), or 64 (two CTAs per SM; narrow lattices waste
                                  less of a tile); 0 with the one-sweep kernel */
    int32_t df_cycles;         /* cycles whose defects were formed in double-float (FP32
                                  pairs, as in a single mixed solve), before the states
                                  were joined and checked in FP64; the rest of the cycles
                                  checked in FP64 */
} rfb_batch_info;

/* hs: n handles (distinct, same device, nx % 4 == 0), not owned; they must outlive the
 * batch. Work is queued on hs[0]'s stream. */
rfb_status rfb_soc_batch_create(rfb_soc_handle* const* hs, int n, rfb_batch** out);

/* Solve every lattice q to residual <= tol[q] at (s_in[q], eta[q]) (host arrays of n).
 * opts (nullable) must select RFB_PREC_MIXED (the default of this call is still the
 * opts default, so pass opts with precision = RFB_PREC_MIXED); velocity_scale, cfl,
 * dt_mode, inlet_bc, max_sweeps (per lattice) and check_every (0 = autotuned) apply to
 * all. opts.fp32_kernel: 0 = the faster of the one-sweep kernel over every lattice and
 * the batched two-sweep TMA pass (local steps only; timed once per batch), 1 = the
 * one-sweep kernel, 2 = the two-sweep pass with the tile width (128 or 64 columns), TMA
 * stage count and z chunk timed, 3..6 = the two-sweep pass with 128-column tiles, 7 / 8 =
 * with 64-column tiles (two CTAs per SM); 2..8 give RFB_ERR_INVALID_ARG with the global
 * step, larger values always. With the two-sweep pass the sweeps per cycle are a multiple
 * of 4. The defects of the cycles are formed in double-float until every lattice has
 * reached its tol or, where tol lies below what double-float defects resolve (10 x tau
 * 2^-44 max_c d_c), that level (info->df_cycles); the states are then joined and checked
 * in FP64, and a lattice above its tol there continues with FP64 checks, so every result
 * is FP64-confirmed (the handles need the memory of a mixed solve: the assembled operator
 * as FP64 and as FP32 pairs, and a double-float state). Each handle warm-starts from its
 * state if it has one. res (nullable, n entries) and info (nullable) are filled. Returns
 * RFB_ERR_NOT_CONVERGED if max_sweeps ran out first; the states of every handle are
 * valid either way. */
rfb_status rfb_soc_batch_solve(rfb_batch* b, const double* s_in, const double* eta,
                               const double* tol, const rfb_solve_opts* opts,
                               rfb_solve_result* res, rfb_batch_info* info);

/* Queue the batch's work on this cudaStream_t (a created stream, not the legacy or
 * per-thread default stream: the cycle is captured into a CUDA graph). By default the
 * batch creates a non-blocking stream of its own. */
rfb_status rfb_soc_batch_set_stream(rfb_batch* b, void* cuda_stream);

/* Last error detail of the batch (b = NULL: of the last failed rfb_soc_batch_create). */
const char* rfb_soc_batch_last_error(const rfb_batch* b);

/* Release the batch (not its handles). NULL-safe. */
rfb_status rfb_soc_batch_destroy(rfb_batch* b);

/* Lattice size N and fluid-cell count of the handle (either pointer nullable). */
rfb_status rfb_soc_info(const rfb_soc_handle* h, int64_t* n_cells, int64_t* n_fluid);

/* Number of CUDA kernels this handle has launched since creation (graph replays count
 * every kernel inside the graph). */
int64_t rfb_soc_kernel_launches(const rfb_soc_handle* h);

/*
 * Nernst model (Sec. II.D, Eqs. nernst-eta-inst-def,
 * nernst-model-eta-update, nernst-model-s-update; explicit form Algorithm 8): the steady
 * state of the SBV problem (the same as rfb_soc_solve's) reached by treating electrode
 * cells (fluid cells with k0 m n_wall / dx > 0) as Dirichlet cells s = sigma(V~ - eta~)
 * with an overpotential field eta~ updated from the transport rate of each step:
 *   eta~_I = 2 asinh(-T / (2 k0 a sqrt(s (1 - s)))),  eta~ <- (1 - w) eta~ + w eta~_I,
 * w = omega / (1 + |G|) per cell, G the slope of this fixed-point map at the cell (a single
 * weight must stay below 2 / (1 + |G|) at every electrode cell; the scaling makes every
 * omega in (0, 1] stable, omega = 1 being the cell's Newton step). Other fluid cells take
 * the explicit pseudo-time step. Convergence is judged by the FP64 residual of the SBV
 * problem, so res holds the same quantities as rfb_soc_solve's. Cold start (no state):
 * s = s_in, eta~ = 0, electrode cells at sigma(V~); warm start: the current state with
 * eta~ = V~ - logit(s). Requirements: kinetics mode 0 with alpha = 1/2 (the sinh form of
 * Eq. source-term-bv), k0 > 0, opts precision RFB_PREC_FP64, 0 < omega <= 1; otherwise
 * RFB_ERR_INVALID_ARG. A converged result allows rfb_soc_adjoint at this operating point.
 */
rfb_status rfb_soc_solve_nernst(rfb_soc_handle* h, double s_in, double overpotential,
                                double tol, double omega, const rfb_solve_opts* opts,
                                rfb_solve_result* res);

/* eta~ of the last rfb_soc_solve_nernst on the current state: N doubles (host or device
 * per kind), 0 off the electrode cells. RFB_ERR_STATE if there is none (reset_state and
 * set_state drop it). */
rfb_status rfb_soc_get_overpotential(rfb_soc_handle* h, double* eta_t, rfb_mem_kind kind);

/* Parameters of the Butler-Volmer model with electromigration (rfb_soc_solve_bv); zero
 * fields take the default in brackets. */
typedef struct rfb_bv_params {
    double D_H;        /* proton diffusivity [m^2/s] (9.3e-9, parameter table) */
    double D_X;        /* HSO4- diffusivity [m^2/s] (1.38e-9; the table's second proton
                          row, read as the counter-ion) */
    double c_H_in;     /* inlet proton concentration [mol/m^3] (50 c0: 1 M sulfuric acid
                          against 20 mM quinone, Sec. II.B) */
    double cg_rtol;    /* each potential solve stops at max|residual| <= cg_rtol
                          max|right-hand side| (1e-13) */
    int32_t cycle;     /* species sweeps between potential solves (100) */
    int32_t max_cg;    /* conjugate-gradient iterations per potential solve (100000) */
    int32_t start;     /* 0: from the handle's converged SBV state at the same operating
                          point when there is one (model refinement, Sec. III.C), else from
                          s = s_in; 1: SBV state required (RFB_ERR_STATE without one);
                          2: from s = s_in */
    int32_t reserved;  /* must be 0 */
} rfb_bv_params;

typedef struct rfb_bv_result {
    int64_t sweeps;          /* species sweeps */
    int64_t cycles;          /* potential solves */
    int64_t cg_iterations;   /* conjugate-gradient iterations, all solves */
    double residual;         /* max over O, R, H of tau RMS(RHS_j) / scale_j, scale c0
                                for the quinones and c_H_in for protons */
    double dphi;             /* largest change of phi in the last potential solve [V] */
    double I_tot;            /* n_e F h^3 sum S [A] (Eq. I-tot-def) */
    double U;                /* I_tot / (n_e F c0 Q (1 - s_in)) (Eq. utilization-def) */
    double s_out;            /* flow-weighted outlet mean of s = C_R / (C_O + C_R) */
    double I_membrane;       /* protons' migration current through the membrane [A] */
    double phi_mean;         /* mean of phi_L over fluid cells [V] */
    double phi_min;          /* smallest phi_L [V] */
    double phi_max;          /* largest phi_L [V] */
    double time_ms;
} rfb_bv_result;

/*
 * Steady state of the Butler-Volmer model with electromigration (Sec. II.C, Eqs.
 * nernst-planck, poisson-phi, kappa, electroneutrality; Algorithm 2 in steady form) on
 * the handle's lattice, flow and kinetics: oxidised and reduced quinone (charge -2,
 * diffusivity D), protons (+1, D_H) and the electrolyte potential phi_L, with HSO4- by
 * electroneutrality. The source is the Butler-Volmer rate with the overpotential of
 * Eq. etat-from-s-bv, k0 a (C_O e^{alpha V_c} - C_R e^{(alpha-1) V_c}),
 * V_c = V~ + n_e phi_L / V_T; O + 2 H+ + 2 e- -> R. Boundaries: inlet concentrations
 * (1 - s_in) c0, s_in c0, c_H_in and zero normal field; zero-gradient outlet; no flux
 * and zero normal field at side walls and fibers; the membrane (phi_L = 0) is the low-x
 * face of the cells i = 0, crossed by protons only (migration, C_H of the cell, half a
 * cell). The potential equation is solved as div(kappa grad phi) with face
 * conductivities from Eq. kappa, as the discrete charge balance of the species fluxes.
 * Species: FP64 explicit pseudo-time sweeps at a fixed potential (local steps, opts.cfl);
 * every bv->cycle sweeps the potential is solved by conjugate gradients on the device.
 * Converged when res->residual <= tol and the last potential solve changed phi by at most
 * tol V_T / n_e and reached its own tolerance (or the rounding floor of its residual; a
 * solve cut off by max_cg does not count). From a cold start (start = 2, or no SBV state)
 * the species first relax at phi = 0 to residual 1e-3. Needs kinetics mode 0,
 * opts.precision FP64, opts.dt_mode local.
 *   bv    nullable (defaults)
 *   res   nullable
 * Returns RFB_OK, RFB_ERR_NOT_CONVERGED (opts.max_sweeps or opts.timeout_ms; the state is
 * valid), RFB_ERR_NONFINITE, RFB_ERR_INVALID_ARG, RFB_ERR_STATE (start = 1 without an SBV
 * state). The SOC state of the handle is not changed; rfb_soc_get_bv_state reads the
 * result.
 */
rfb_status rfb_soc_solve_bv(rfb_soc_handle* h, double s_in, double overpotential, double tol,
                            const rfb_bv_params* bv, const rfb_solve_opts* opts,
                            rfb_bv_result* res);

/* The last rfb_soc_solve_bv state: C_O, C_R, C_H [mol/m^3] and phi_L [V], N doubles each
 * (host or device per kind; any pointer may be NULL), 0 on solid cells. RFB_ERR_STATE if
 * there is none. */
rfb_status rfb_soc_get_bv_state(rfb_soc_handle* h, double* c_o, double* c_r, double* c_h,
                                double* phi, rfb_mem_kind kind);

/* Self-test of the bounded waits of the two-sweep pass (no counterpart in the paper):
 * launches one block on the current device that waits, through the same bounded
 * mbarrier wait as the pass, on a barrier nothing completes, polling at most spin_limit
 * times (1 .. 2^26). *gave_up = 1 when every thread gave up, recorded the error and the
 * kernel ran to its end (the context stays usable). RFB_ERR_INVALID_ARG for a bad
 * argument, RFB_ERR_CUDA if a CUDA call failed (detail in rfb_soc_last_error(NULL)). */
rfb_status rfb_selftest_bounded_wait(int64_t spin_limit, int32_t* gave_up);

/* The FP32 correction kernel the handle's autotuner chose for RFB_PREC_MIXED solves with
 * fp32_kernel = 0 or 2 (or the one a solve forced), as an opts.fp32_kernel value: 0 = not
 * chosen yet, 1 = one sweep per launch, 3 / 4 = two-sweep passes in the persistent /
 * chunked launch shape, 5 / 6 the same with four TMA stages, 7 .. 10 three-sweep passes;
 * and the timed device milliseconds per sweep of the one-sweep kernel and of the fastest
 * pass variant (0 if not timed). Any output pointer may be NULL. */
rfb_status rfb_soc_tuned_fp32_kernel(const rfb_soc_handle* h, int32_t* kernel,
                                     double* plain_ms_per_sweep,
                                     double* blocked_ms_per_sweep);

#ifdef __cplusplus
}
#endif

#endif /* RFB_SOC_H */
