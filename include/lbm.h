/*
 * lbm.h -- C ABI of the GB300 implementation of the fused collide-and-stream
 * step of the modified lattice BGK model for convection heat transfer in
 * porous media (Wang, Mi and Guo, arXiv 1505.02976).
 *
 * One time step advances two D2Q9 distributions on an nx x ny lattice:
 *   flow:     f_i(x + c_i, t + 1) = f_i - (f_i - f_i^eq)/tau_f + F_i   (Eq. LBEeq)
 *   thermal:  g_i(x + c_i, t + 1) = g_i - (g_i - g_i^eq)/tau_T + P_i + Q_i
 *                                                       (Eqs. LBEHeq, TEqColli)
 * with the porous equilibrium of Eqs. (EQFIN)-(EQTSHIN), the Guo forcing term
 * of Eq. (FtermF) carrying the Brinkman-Forchheimer force of Eq. (ForceEq),
 * the modified thermal equilibrium and sources of Eqs. (TeEDFEQ), (Eq:Tforce),
 * the local shear-rate and temperature-gradient schemes of Sec. 3.3
 * (Eqs. ShearEqCom, TeEqCom) and the non-equilibrium extrapolation walls of
 * Sec. 3.4 (Eqs. NEESVel, TNEESAp, TNEESApGra), all fused into one kernel
 * launch per step.  Lattice units throughout: dx = dt = 1, c_s^2 = 1/3.
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 * Layout of fields passed in or out: row-major [ny][nx] (x fastest), float64.
 * Layout of population arrays passed in or out: [9][ny][nx] float64, index i
 *   in the paper's velocity order (Sec. 3.1): 0 rest, 1 (+1,0), 2 (0,+1),
 *   3 (-1,0), 4 (0,-1), 5 (+1,+1), 6 (-1,+1), 7 (-1,-1), 8 (+1,-1).
 * Sides: 0 = W (x = 0), 1 = E (x = nx-1), 2 = S (y = 0), 3 = N (y = ny-1).
 *   Wall nodes are the outermost nodes; the characteristic length defaults to
 *   L = nx - 1.
 * on_device: 0 = the pointers are host memory (the call copies through a
 *   device staging area and returns after the copy; input fields in
 *   page-locked host memory are instead read in place by the kernel that
 *   consumes them, and the call returns once it has); 1 = the pointers are
 *   device memory of the handle's device (the call is asynchronous on the
 *   handle's stream).
 * Ownership: the caller owns every pointer it passes; nothing is retained
 *   after a call returns.  The handle owns its device state, which lives in
 *   the workspace (caller-provided or allocated by lbm_create).
 * Errors: every entry point returns an lbm_status; no exception or abort
 *   crosses the ABI.  lbm_last_error() gives a message for the last failure.
 *   LBM_ERR_NONFINITE and LBM_ERR_TIMEOUT are sticky until lbm_set_fields
 *   or lbm_set_state.
 * Threading: a handle must not be used from two threads at once.
 */
#ifndef LBM_GB300_H
#define LBM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_handle lbm_handle;

typedef enum {
    LBM_OK = 0,
    LBM_ERR_ARG = -1,          /* bad pointer, size, side or flag */
    LBM_ERR_CUDA = -2,         /* a CUDA runtime call failed */
    LBM_ERR_NONFINITE = -3,    /* a NaN/Inf appeared in u or T during a step */
    LBM_ERR_TIMEOUT = -4,      /* a bounded device-side wait gave up */
    LBM_ERR_PARAM_RANGE = -5,  /* parameters outside the model's range (Sec. 4) */
    LBM_ERR_OOM = -6,          /* workspace too small or allocation failed */
    LBM_ERR_GUARD = -7         /* a guard word of the workspace was overwritten */
} lbm_status;

/* Storage type of the populations.  LBM_F64 computes in FP64, LBM_F32 and
 * LBM_F16 in FP32; all store the flow populations f_1..f_8 as they are and
 * the thermal populations as deviations g_i - w_i sigma T0 from the rest
 * state.  LBM_F16 stores them scaled by 2^10 and rounded stochastically
 * (rounded up with probability equal to the discarded fraction, random bits
 * from a counter-based hash of the node pair and the step), so that every
 * stored value is exact in expectation. */
typedef enum { LBM_F64 = 0, LBM_F32 = 1, LBM_F16 = 2 } lbm_precision;

/* Boundary kind of one side. */
typedef enum {
    LBM_BC_PERIODIC = 0,   /* periodic; the opposite side must be periodic too */
    LBM_BC_DIRICHLET = 1,  /* no-slip (velocity u_bc) and prescribed T = T_bc */
    LBM_BC_ADIABATIC = 2   /* no-slip (velocity u_bc) and dT/dn = 0 */
} lbm_bc;

/* Problem statement, in the paper's dimensionless groups (Sec. 2, Sec. 4).
 * The fields marked "NaN = derive" are derived when they hold NaN:
 *   L      = nx - 1
 *   U      = Ma c_s                       (characteristic velocity, Sec. 4)
 *   gbeta  = U^2 / ((Th - Tc) L)          (U^2 = g beta dT L)
 *   nu     = U L sqrt(Pr / Ra)            (Ra, Pr of Sec. 2); when A is given
 *            instead, nu = c_s^2 (tau_f - A - 1/2) / J
 *   alpha_e= nu / Pr; when B is given instead, sigma c_s^2 (tau_T - B - 1/2)
 *   A      = tau_f - 1/2 - J nu / c_s^2   (Eq. EQA&B for J = 1)
 *   B      = tau_T - 1/2 - alpha_e / (sigma c_s^2)
 *   K      = Da L^2                       (Sec. 2)
 * F_eps = 1.75 / sqrt(150 eps^3) (Ergun) when forchheimer = 1, else 0.
 *   T0     = (Th + Tc) / 2                (buoyancy reference and thermal rest
 *            state; the heat-generating cavity of Sec. 4.3 puts it at T_c)
 *   Q      = Ra_I alpha_e (Th - Tc) / (Ra L^2)   (internal heat source,
 *            Sec. 4.4; with Ra = Ra_I and Th - Tc = Q L^2 / alpha_e it is the
 *            scaling of Sec. 4.3)
 * Th - Tc normalises the Nusselt number. */
typedef struct {
    int32_t nx, ny;          /* nodes, wall nodes included; >= 4 across walls */
    int32_t bc[4];           /* lbm_bc per side W, E, S, N */
    int32_t forchheimer;     /* 1: Ergun F_eps, 0: no quadratic drag */
    int32_t da_infinite;     /* 1: K = infinity (no Darcy/Forchheimer drag) */
    int32_t precision;       /* lbm_precision */
    int32_t moment_state;    /* 1: store the moment state (tau_f = tau_T = 1; see below) */
    double Ra, Pr, Da, J, eps, sigma, Ma;
    double tau_f, tau_T;
    double Th, Tc, T_init, rho0, Q, ax, ay;
    double L, nu, alpha_e, gbeta, A, B, K;   /* NaN = derive */
    double T_bc[4];          /* Dirichlet wall temperature per side */
    double u_bc[4][2];       /* wall velocity per side */
    double T0;               /* NaN = derive */
    double Ra_I;             /* internal Rayleigh number (used when Q is NaN) */
} lbm_params;

/* Moment state (moment_state = 1).  At tau_f = tau_T = 1 the collision
 * leaves f* = f^eq + F_i and g* = g^eq + P_i + Q_i (Eqs. LBEeq, TEqColli),
 * functions of the nine numbers (p, u, S, T, grad T) that a step computes
 * for every node (wall nodes: their boundary state, Sec. 3.4).  The handle
 * then stores those nine moments per node instead of the 17 populations and
 * each step rebuilds the populations in on-chip memory; the results are the
 * same as with population storage up to rounding.  Requires tau_f = tau_T = 1
 * and LBM_F32 or LBM_F64 (else LBM_ERR_ARG).  lbm_set_state and lbm_adjoint
 * need population storage and return LBM_ERR_ARG on such a handle; every
 * other call behaves as with populations (lbm_get_state returns the
 * post-collision populations the moments define). */

/* Row segments per column band of the moment-state step (segments >= 1;
 * 0 restores the default, which fills the GPU's resident blocks once).
 * Every choice computes the same values.  LBM_ERR_ARG on a population
 * handle. */
lbm_status lbm_set_moment_segments(lbm_handle* h, int32_t segments);

/* Step kernel of a population handle (no counterpart in the paper; a
 * launch choice).  FP32 and FP16 lattices walled on all four sides default
 * to staged rows: each block loads the 17 planes its rows pull from into
 * shared memory with tensor copies and waits on them with bounded waits.
 * staged = 0 selects the kernel in which every thread loads its own 17
 * values from global memory; staged = 1 restores the staged kernel
 * (LBM_ERR_ARG where it is unavailable: FP64, a periodic side, the moment
 * state, a lattice under 4 x 4, or a CUDA driver without tensor-map encoding).
 * Both kernels run the same per-node arithmetic (results agree to rounding;
 * bit for bit in FP32 at tau_f = tau_T = 1).  In FP16 at tau_f = tau_T = 1
 * the staged kernel computes pairs of interior nodes with packed FP32
 * instructions, whose fused multiply-adds can round differently: its stored
 * values then agree with the other kernel's to within one FP16 rounding
 * step plus FP32 rounding.  lbm_step_staged returns 1 when the next step
 * uses staged rows, else 0. */
lbm_status lbm_set_step_staging(lbm_handle* h, int32_t staged);
int32_t lbm_step_staged(const lbm_handle* h);

/* Fill p with the paper's defaults (Sec. 4): the 32 x 32 porous cavity,
 * hot W wall T = 1, cold E wall T = 0, adiabatic S and N, no slip, rho0 = 1,
 * J = sigma = 1, tau_f = tau_T = 1, Ma = 0.1, Ra = 1e3, Da = 1e-2,
 * eps = 0.6, Pr = 1, Forchheimer on, T_init = 0.5, FP32 storage. */
lbm_status lbm_params_default(lbm_params* p);

/* Derived lattice constants of p, in this order:
 * L, T0, dT, U, gbeta, nu, nu_e, alpha_e, A, B, K, F_eps, Q (13 doubles).
 * Returns LBM_ERR_PARAM_RANGE when the parameters are outside the range the
 * model admits: 0 < eps <= 1, tau > 1/2, A < tau_f - 1/2, B < tau_T - 1/2
 * (Sec. 4), sigma > 0, rho0 > 0. */
lbm_status lbm_derived(const lbm_params* p, double out[13]);

/* Bytes of device workspace a handle for p needs (two population buffers,
 * field staging, reduction scratch, residual snapshot). */
lbm_status lbm_workspace_size(const lbm_params* p, size_t* bytes);

/* Create a handle.  stream: a cudaStream_t (NULL = the legacy default
 * stream).  workspace: device memory of at least lbm_workspace_size() bytes
 * aligned to 256 bytes, owned by the caller and kept alive until
 * lbm_destroy; NULL = the library allocates it (cudaMalloc) and frees it in
 * lbm_destroy.  The lattice starts at the uniform rest state
 * (u = 0, p = 0, T = T_init): call lbm_set_fields to change it. */
lbm_status lbm_create(const lbm_params* p, void* stream, void* workspace,
                      size_t workspace_bytes, lbm_handle** out);

void lbm_destroy(lbm_handle* h);

/* Message of the last failure on h (or of the last failed lbm_create when h is
 * NULL).  Valid until the next call on h. */
const char* lbm_last_error(const lbm_handle* h);

/* Initialise the state from macroscopic fields: the post-collision
 * populations become f = f^eq(p = 0, u, S = 0) and
 * g = g^eq(T, u, p = 0, grad T = 0) (Eqs. EQFIN, TeEDFEQ).  Any of T, ux, uy
 * may be NULL (T_init, 0, 0).  eps_field: a porosity field [ny][nx] with
 * values in (0, 1), or NULL for the uniform porosity eps.  With a field, the
 * permeability of each node follows the Kozeny-Carman form of the Ergun
 * relation (Sec. 2), K(e) = Da L^2 [e^3/(1-e)^2] / [eps^3/(1-eps)^2] with
 * the problem's eps as the reference (which must then be below 1), and
 * F_eps(e) = 1.75/sqrt(150 e^3).  Resets the step counter and the non-finite
 * flag. */
lbm_status lbm_set_fields(lbm_handle* h, const double* T, const double* ux,
                          const double* uy, const double* eps_field,
                          int on_device);

/* Stream function of the current velocity field (the u_x of lbm_moments):
 * u_x = d psi / dy, psi = 0 along the row y = 0, integrated up each column
 * by the trapezoid rule, psi(x, y) = psi(x, y - 1) + (u_x(x, y - 1) +
 * u_x(x, y)) / 2 in lattice units.  The paper reports the extreme of psi
 * (Sec. 4.3, Table 3, normalised there by L sqrt(g beta dT L)) without
 * stating its discretisation.  psi: nx * ny doubles [y][x], host or device
 * (on_device), or NULL; range: host array receiving min and max of psi, or
 * NULL.  Host outputs: the call synchronises. */
lbm_status lbm_stream_function(lbm_handle* h, double* psi, int on_device, double range[2]);

/* External acceleration profile: a_y(y) = ay[y] is added to the uniform a_y
 * of the parameters in G = g beta (T - T0) j + a (Sec. 2), one value per
 * row y = 0..ny-1, host memory (copied; NULL removes the profile).  The
 * mixed-convection channel of Sec. 4.1 is driven by such a profile.
 * Synchronises. */
lbm_status lbm_set_force_profile(lbm_handle* h, const double* ay);

/* Advance n >= 0 time steps (stream, rebuild walls, collide; one kernel
 * launch per step).  Asynchronous on the handle's stream.  Returns
 * LBM_ERR_NONFINITE or LBM_ERR_TIMEOUT if an earlier synchronising call saw
 * the corresponding flag.  FP32 lattices walled on all four sides stage the
 * pulled rows in shared memory with tensor copies and bounded waits. */
lbm_status lbm_step(lbm_handle* h, int64_t n);

/* Wait for the handle's stream; returns LBM_ERR_TIMEOUT if a bounded
 * device-side wait of a step gave up (the state is then undefined), else
 * LBM_ERR_NONFINITE if any step since the last reset produced a non-finite
 * velocity or temperature. */
lbm_status lbm_sync(lbm_handle* h);

/* Out-of-bounds detection (the paper has no counterpart): every region of
 * the handle's workspace (population or moment buffers, fields, snapshot,
 * scratch) is followed by 256 guard bytes of 0xA5, written by lbm_create.
 * Synchronises the stream and compares them; LBM_ERR_GUARD names the first
 * overwritten guard (a kernel wrote past the end of the region before it).
 * The workspace size reported by lbm_workspace_size includes the guards. */
lbm_status lbm_check_guards(lbm_handle* h);

/* Failure-detection self-test (the paper has no counterpart): launches, on
 * the handle's stream, one kernel whose bounded device-side wait cannot
 * succeed (an mbarrier that nothing arrives on, 20 ms limit); it gives up
 * and raises the handle's timeout flag, so the next lbm_sync returns
 * LBM_ERR_TIMEOUT and the context stays usable.  lbm_set_fields or
 * lbm_set_state clear the status.  Asynchronous. */
lbm_status lbm_wait_selftest(lbm_handle* h);

/* FP64 throughput of the device (the paper has no counterpart; a
 * measurement helper): runs, on the given stream (a cudaStream_t, NULL = the
 * legacy default stream), a kernel of independent FP64 fused multiply-add
 * chains filling every SM, times it with CUDA events and stores the rate in
 * FLOP/s (one FMA = 2 FLOP) in *flops_per_s (host).  The FP64 step is bound
 * by this rate, not by memory; it is the denominator of that step's
 * roofline.  Synchronises the stream; LBM_ERR_CUDA on any CUDA failure. */
lbm_status lbm_fp64_peak(void* stream, double* flops_per_s);

/* Macroscopic fields of the current state: the pressure, velocity and
 * temperature that the next step computes after streaming (Sec. 3.1-3.2);
 * wall nodes report their boundary state (u_b, T_b, p(x_f)) of Sec. 3.4.
 * Any output may be NULL.  Host outputs: the call synchronises. */
lbm_status lbm_moments(lbm_handle* h, double* p, double* ux, double* uy,
                       double* T, int on_device);

/* Average Nusselt number on one wall (Eq. Eq:AvNuss):
 * Nu(s) = -L (dT/dn) / (Th - Tc), the derivative along +x (W, E walls) or +y
 * (S, N walls) taken by the second-order one-sided difference from the wall
 * node inward; the mean is the trapezoid rule over the wall's nodes divided
 * by (number of nodes - 1).  Temperatures are taken in FP64 from the stored
 * populations.  nu_local (NULL allowed) receives ny (W, E) or nx (S, N)
 * values, in host memory.  Synchronises. */
lbm_status lbm_nusselt(lbm_handle* h, int side, double* nu_mean, double* nu_local);

/* Mean Nusselt number of one wall, as lbm_nusselt computes it, for callers
 * that must not allocate device memory (a program that reserves its whole
 * device budget itself, a plugin that may not grow its host's footprint, a
 * loop that cannot take the device-wide synchronisation of cudaMalloc).
 * The paper has no counterpart to this entry point.  It allocates nothing:
 * the per-node values live in a fixed array compiled into the library (held
 * on every GPU that loads it until exit), so the wall may have at most 65536
 * nodes (else LBM_ERR_ARG).  Every call looks up that array's device
 * address on the device of the handle's stream.  All calls share the array:
 * calls whose GPU work overlaps (other streams or other handles on the same
 * device) race.  nu_mean: host pointer.  Synchronises the handle's stream. */
lbm_status lbm_nusselt_noalloc(lbm_handle* h, int side, double* nu_mean);

/* Steady-state criterion of Sec. 4 against the snapshot taken by the
 * previous lbm_residual call (or lbm_set_fields):
 *   res_u = sum |u - u_old|_2 / sum |u|_2,  res_T = sum |T - T_old| / sum |T|,
 * reduced in FP64 in a fixed order (deterministic), then the snapshot is
 * replaced by the current fields.  Synchronises. */
lbm_status lbm_residual(lbm_handle* h, double* res_u, double* res_T);

/* Totals of the stored post-collision state, reduced in FP64 in a fixed
 * order: sum_f = sum over nodes of f_1 + ... + f_8 (f_0 is not stored),
 * sum_g = sum over nodes of g_0 + ... + g_8.  With periodic sides and Q = 0
 * sum_g is conserved exactly by the step (sum_i g_i^eq = sigma T and
 * sum_i P_i = 0, Sec. 3.2): the energy diagnostic.  Synchronises. */
lbm_status lbm_totals(lbm_handle* h, double* sum_f, double* sum_g);

/* The post-collision populations of the last step as float64 [9][ny][nx]
 * arrays, g absolute (not as a deviation).  f_0 is not stored by the GPU
 * path (no moment reads it: p uses sum_{i!=0} f_i, Sec. 3.1) and is
 * reported as NaN. */
lbm_status lbm_get_state(lbm_handle* h, double* f, double* g, int on_device);

/* Load post-collision populations (layout of lbm_get_state; f_0 ignored).
 * Resets the non-finite flag; keeps the step counter. */
lbm_status lbm_set_state(lbm_handle* h, const double* f, const double* g, int on_device);

/* Discrete adjoint of the hot-wall heat transfer.  From the current state,
 * advance n_steps steps (the handle ends at step n_steps), evaluate
 * loss = mean Nusselt number on `side` (as lbm_nusselt, with Th - Tc held at
 * its nominal value), then run the adjoint of every step backwards and return
 *   dloss_deps[ny][nx]  d loss / d eps at every node (host; NULL allowed;
 *                       needs a porosity field set by lbm_set_fields),
 *   dloss_dTbc[4]       d loss / d (Dirichlet wall temperature) per side
 *                       W, E, S, N (host; NULL allowed).
 * States are recomputed from checkpoints kept every `segment` steps
 * (0 = ceil(sqrt(n_steps))): memory for about 2 sqrt(n_steps) states is
 * allocated on the handle's stream for the duration of the call and freed
 * before it returns.  FP64 or FP32 storage; the adjoint arithmetic is that of
 * the storage type, the gradients are accumulated in FP64.  The derivatives
 * are those of the discrete step itself (each node's transposed Jacobian is
 * applied exactly, with the transpose of the streaming), not of the
 * continuous equations.  The paper has no adjoint; the loss and the
 * parameters are those of its cavity problem (Sec. 4.2).  Synchronises. */
lbm_status lbm_adjoint(lbm_handle* h, int64_t n_steps, int64_t segment, int side, double* loss,
                       double* dloss_deps, double* dloss_dTbc);

/* Save (save = 1) or restore (save = 0) the complete state: populations,
 * porosity field and step counter.  The file holds a header (format tag,
 * precision, lattice shape, a hash of the lbm_params the handle was created
 * with), the raw stored planes and a CRC-32 of them; a restore checks all of
 * them on the host before it touches the device and fails with LBM_ERR_ARG
 * on any mismatch or corruption, leaving the state unchanged.  (A CUDA
 * failure while the checked payload is copied to the device returns
 * LBM_ERR_CUDA and leaves the state undefined.)  A restored run continues
 * bit for bit as the saved one would have.  Neither the force profile of
 * lbm_set_force_profile nor the residual snapshot is part of the file: set
 * the profile again on the restoring handle; the restored state becomes the
 * reference of the next lbm_residual.  Synchronises. */
lbm_status lbm_checkpoint(lbm_handle* h, const char* path, int save);

/* Steps completed since the last lbm_set_fields. */
int64_t lbm_steps_done(const lbm_handle* h);

/* Number of step-kernel launches issued by this handle so far. */
int64_t lbm_kernel_launches(const lbm_handle* h);

/* ------------------------------------------------------------------------
 * Batches: many independent cavities of different size and parameters
 * advanced together (the paper's cavity problem of Sec. 4.2 run for a set of
 * (N, Ra, Da, eps) at once).  Each cavity is the lattice an lbm_params
 * describes; all cavities of a batch share the storage precision (FP64 or
 * FP32) and step together.  The state of every cavity starts at its uniform
 * rest state.
 * ---------------------------------------------------------------------- */
typedef struct lbm_batch lbm_batch;

typedef enum {
    LBM_BATCH_FUSED = 0,     /* one kernel launch per step for all cavities */
    LBM_BATCH_GRAPH = 1,     /* the same launches replayed from a captured CUDA graph
                                (50 steps per graph; needs a non-default stream) */
    LBM_BATCH_PER_CASE = 2,  /* one single-lattice launch per cavity per step */
    LBM_BATCH_PERSISTENT = 3 /* every step of the call in one cooperative launch: each resident
                                block keeps taking (cavity, band, segment) items and waits,
                                bounded, only until the item's neighbours have finished the
                                previous step (staged batches only, else LBM_ERR_ARG) */
} lbm_batch_mode;

/* Bytes of device workspace for the n cavities of p[0..n-1]. */
lbm_status lbm_batch_workspace_size(const lbm_params* p, int32_t n, size_t* bytes);

/* Create a batch of the n cavities p[0..n-1] (same conventions as
 * lbm_create: caller workspace or NULL for a library allocation). */
lbm_status lbm_batch_create(const lbm_params* p, int32_t n, void* stream, void* workspace,
                            size_t workspace_bytes, lbm_batch** out);

void lbm_batch_destroy(lbm_batch* b);

const char* lbm_batch_last_error(const lbm_batch* b);

/* Initialise cavity `cavity` from host fields [ny][nx] (NULL: T_init, 0, 0),
 * as lbm_set_fields does; cavity = -1 resets every cavity to its rest state
 * (fields must then be NULL) and the step counter.  Synchronises. */
lbm_status lbm_batch_set_fields(lbm_batch* b, int32_t cavity, const double* T, const double* ux,
                                const double* uy);

/* Advance every cavity n steps in the given lbm_batch_mode.  Asynchronous. */
lbm_status lbm_batch_step(lbm_batch* b, int64_t n, int mode);

/* Pick the tile width (32, 64 or 128 nodes; tiles hold 128 nodes) and the
 * grid size (1, 2 or 4 waves of resident blocks) of the fused step by timing
 * steps_per_candidate + 1 steps of each candidate.  These are real steps of
 * the run (every launch shape computes identical values).  The launch shape
 * belongs to the global-load kernel; a staged batch (below) times the same
 * kernel for every candidate.  Synchronises. */
lbm_status lbm_batch_autotune(lbm_batch* b, int32_t steps_per_candidate, int32_t* tile_x, int32_t* grid);

/* Set the fused step's launch shape explicitly (global-load kernel). */
lbm_status lbm_batch_set_launch(lbm_batch* b, int32_t tile_x, int32_t grid);

/* Step kernel of a batch (no counterpart in the paper; a launch choice).
 * A batch of FP32 cavities that are all walled on all four sides (each at
 * least 4 x 4) defaults to staged rows: one block per band of 128 columns x
 * 4 rows of one cavity loads the planes its rows pull from with tensor
 * copies (the maps of every cavity live in the workspace) and waits on them
 * with bounded waits, in every mode (per-case mode launches the single-
 * lattice staged kernel per cavity).  staged = 0 selects the global-load
 * kernel and its launch shape; staged = 1 restores staging (LBM_ERR_ARG
 * where it is unavailable).  Both run the same per-node arithmetic (bit for
 * bit at tau_f = tau_T = 1).  lbm_batch_staged returns 1 when the next
 * step uses staged rows, else 0. */
lbm_status lbm_batch_set_staging(lbm_batch* b, int32_t staged);
int32_t lbm_batch_staged(const lbm_batch* b);

/* Wait for the stream; LBM_ERR_TIMEOUT if a bounded wait of the staged
 * kernel gave up, else LBM_ERR_NONFINITE if any cavity produced a NaN/Inf
 * (both sticky until lbm_batch_set_fields). */
lbm_status lbm_batch_sync(lbm_batch* b);

/* Mean Nusselt number of every cavity on one side (as lbm_nusselt), into
 * nu_mean[n] in host memory.  Synchronises. */
lbm_status lbm_batch_nusselt(lbm_batch* b, int side, double* nu_mean);

/* Macroscopic fields of one cavity (as lbm_moments), host outputs.
 * Synchronises. */
lbm_status lbm_batch_moments(lbm_batch* b, int32_t cavity, double* p, double* ux, double* uy,
                             double* T);

int64_t lbm_batch_steps_done(const lbm_batch* b);

/* Kernel launches issued for steps (a graph replay counts its 50 launches). */
int64_t lbm_batch_kernel_launches(const lbm_batch* b);

/* As lbm_check_guards, for the batch workspace (both population buffers,
 * descriptors, work lists, tensor maps, fields and scratch). */
lbm_status lbm_batch_check_guards(lbm_batch* b);

#ifdef __cplusplus
}
#endif

#endif /* LBM_GB300_H */
