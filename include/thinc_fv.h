/*
 * thinc_fv.h -- C ABI of the GB300 All-Mach THINC-TDU finite-volume stage
 * (Jiao, Schmidt & Adams, arXiv 2304.00140).
 *
 * One explicit low-storage Runge-Kutta stage (Sec. 3.1, Algorithm 1) of the
 * single-fluid four-equation model (Sec. 2.1, Eq. 2-1/2-2) on structured
 * Cartesian grids: boundary update, primitive/thermodynamic update
 * (App. A, App. B), discontinuity sensor (App. D, Eq. D.4), face
 * reconstruction switching between limited MUSCL (Sec. 3.3, Table 4.2),
 * THINC (Eq. 3-3/3-4) and 4th-order central (Eq. D.1-D.3), the
 * thermodynamic-dependent update of rho and e (Eq. 3-5/3-6), the all-Mach
 * Riemann flux (Eq. 3-1/3-2; Eq. D.5/D.6), the viscous stress and heat
 * conduction fluxes (Eq. 2-2, mixture viscosity Eq. 2-8), the CSF
 * surface-tension source with Gaussian-smoothed curvature (Sec. 3.5,
 * Eq. 3-9/3-10), the gravity source (Eq. 2-2) and the flux-divergence /
 * LSRK register update.  All arithmetic runs in CUDA
 * kernels for sm_103a; there is no CPU path.
 *
 * Conventions
 *   - State arrays are structure-of-arrays, float64, interior cells only,
 *     [nv][nz][ny][nx] with x fastest.  nv = ndim + 2 + (ncomp - 1):
 *       conserved  q = (rho, rho u_0..rho u_{d-1}, rho E, rho Y_0..rho Y_{N-2})
 *       primitive  W = (u_0..u_{d-1}, p, T, Y_0..Y_{N-2})
 *     The last component's mass fraction is 1 - sum of the others.
 *   - Units SI.  2D grids have n[2] = 1.
 *   - A context may hold several independent cases (a batch); per-case calls
 *     take the case index, whole-context calls act on every case.
 *   - Every call returns an fv_status and never aborts.  Host buffers stay
 *     owned by the caller; device memory belongs to the context (allocated
 *     with cudaMalloc, or carved from a caller-provided device workspace).
 *   - Calls are asynchronous on the context's stream except where stated.
 */
#ifndef THINC_FV_H
#define THINC_FV_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FV_MAX_COMP 3
#define FV_MAX_VAR 10

typedef enum {
    FV_OK = 0,
    FV_ERR_ARG = 1,          /* invalid argument or unsupported combination */
    FV_ERR_ALLOC = 2,        /* device memory could not be allocated */
    FV_ERR_CUDA = 3,         /* a CUDA runtime call failed (see fv_last_error) */
    FV_ERR_EOS_NONCONV = 4,  /* closure iteration did not converge */
    FV_ERR_NONPHYSICAL = 5,  /* rho <= 0, p + pinf <= 0, T <= 0 or NaN met in a kernel */
    FV_ERR_STATE = 6         /* call out of order (e.g. step before set_state) */
} fv_status;

enum { FV_BC_PERIODIC = 0, FV_BC_REFLECT = 1, FV_BC_OUTFLOW = 2, FV_BC_INFLOW = 3 };
enum { FV_SG = 0, FV_PR = 1, FV_BARO = 2 };
enum { FV_MINMOD = 0, FV_KOREN = 1, FV_VANLEER = 2, FV_VANALBADA = 3,
       FV_CHAKRAVARTHY = 4, FV_MC = 5, FV_SUPERBEE = 6 };
enum { FV_FP64 = 0, FV_MIXED = 1 };
enum { FV_CONSERVED = 0, FV_PRIMITIVE = 1 };
enum { FV_DIAG_TOTALS = 0,   /* double[nv]: compensated sums of q over the case */
       FV_DIAG_DT = 1,       /* double: last step's dt of the case */
       FV_DIAG_TIME = 2,     /* double: accumulated time of the case */
       FV_DIAG_ERROR = 3,    /* int: device error word (bit set of FV_ERRBIT_*) */
       FV_DIAG_TILE = 4 };   /* double[12]: stage-kernel tile x, y, z, threads chosen by the
                                autotuner (runs it if not yet run; for the fused 2D
                                kernel: strip width, rows per work item, 1, threads),
                                [4..7] the tuner's milliseconds per tile (0 if not
                                timed), [8] 1 if the fused 2D kernel was chosen, 2 for
                                the z-marching 3D kernel (tile x, y, planes per item,
                                threads in [0..3]), [9] its best tuned milliseconds,
                                [10] the primitive pass's, [11] its variant (-1: tiled) */
enum { FV_DIAG_FLAGS = 5 };  /* unsigned char[n cells]: App. D sensor flag f (Eq. D.4) of each
                                interior cell for the current state (x fastest); needs the
                                App. D switch (FV_ERR_ARG otherwise); synchronous; call it
                                between steps, not between the stages of a step (it uses a
                                stage register as scratch) */
enum { FV_ERRBIT_NONPHYS = 1, FV_ERRBIT_NONCONV = 2,
       FV_ERRBIT_TIMEOUT = 4 };   /* a bounded wait in a kernel gave up (reported as FV_ERR_CUDA) */

/* Grid of one case.  lo/hi are the box corners (m); bc[d][0] is the low
 * side of dimension d.  FV_BC_INFLOW is accepted on the x-low side only:
 * inside the disc (in_yc, in_zc, in_radius) the ghost cells take Dirichlet
 * u (in_u, or in_u0 when in_u is NULL), T = in_T and Y = in_Y with
 * zero-gradient p; outside it they are a slip wall. */
typedef struct {
    int ndim;                    /* 2 or 3 */
    int n[3];                    /* interior cells per dimension (n[2] = 1 in 2D) */
    double lo[3], hi[3];
    int bc[3][2];
    double in_yc, in_zc, in_radius, in_T;
    double in_u0[3];
    double in_Y[FV_MAX_COMP];
    const double* in_u;          /* host [3][nz][ny] inflow velocity or NULL; copied at init */
} fv_grid;

/* One material.  FV_SG: stiffened gas p = (gamma-1) rho (e-q) - gamma pinf
 * (Eq. A.1.1; ideal gas when pinf = 0).  FV_PR: Peng-Robinson (Eq. A.2.1)
 * with constant ideal-gas cv; M is the molar mass in kg/mol.  FV_BARO: the
 * barotropic model of Sec. 2.2 -- the component at fv_components.liquid is
 * the liquid / liquid-vapour mixture with saturation pressure psat,
 * saturated liquid and vapour densities rho_sl, rho_sv and liquid sound
 * speed cl (Eq. 2-3, 2-4, 2-7), every other one an ideal gas at a fixed
 * temperature with rt = R T_ref (Eq. 2-5).  Then p = f(rho, Y) and the energy
 * is carried passively: the T slot of primitive states holds the specific
 * internal energy e.  All components share one kind.  mu (Pa s) and
 * kc (W/(m K)) are the dynamic viscosity and thermal conductivity of the
 * stress and heat-flux terms of Eq. 2-2, mixed by volume fraction (Eq. 2-8,
 * no vapour); 0 for every component = inviscid.  Viscous terms need
 * stiffened-gas / ideal-gas components (FV_ERR_ARG otherwise). */
typedef struct {
    int kind;
    double gamma, pinf, cv, q;
    double Tc, pc, omega, M;
    double mu, kc;
    double psat, rho_sl, rho_sv, cl, rt;
} fv_component;

typedef struct {
    int ncomp;                   /* 2 or 3 */
    int liquid;                  /* component whose volume fraction feeds CSF and the gas sensor */
    fv_component comp[FV_MAX_COMP];
} fv_components;

/* Closure options and scheme switches ("eos" = closure + scheme). */
typedef struct {
    int iles;                    /* 0: plain (upwind/THINC everywhere), 1: App. D central switch */
    int thinc;                   /* THINC for mass fractions on eligible cells (Sec. 3.3) */
    double beta, thinc_eps, thinc_gamma;   /* beta of Eq. 3-3; eligibility eps; guard gamma */
    int lim_vel, lim_scalar;     /* FV_* limiter ids for velocities and for p, T, Y */
    double thr_ducros, thr_gas, eps_ducros, d3p_coef;   /* Eq. D.4 thresholds, D.5 scale */
    double sigma;                /* surface tension coefficient (N/m); 0 disables CSF */
    double grad_eps;             /* |grad alpha~| * dx below this gives a zero normal */
    int precision;               /* FV_FP64 or FV_MIXED */
    double p_ref, T_ref;         /* offsets carried by the FP32 arithmetic of FV_MIXED */
    double gravity[3];           /* body force per unit mass (m/s^2) of Eq. 2-2: source rho g
                                    (momentum) and rho u . g (energy); zero = off */
    double thr_vap;              /* App. D vapour-fraction sensor threshold (FV_BARO) */
    int curvature;               /* CSF curvature: 0 vertex normals of the Gaussian-smoothed
                                    fraction (Sec. 3.5, Eq. 3-9/3-10), 1 the height function
                                    of 5-cell columns (the Sec. 3.5 option) */
    int st_model;                /* surface tension model: 0 the CSF volume force sigma kappa
                                    grad(alpha) (Sec. 2.3, 3.5); 1 the capillary pressure jump
                                    [P] = sigma kappa [alpha] inside the Riemann solver (the
                                    Sec. 3.5 alternative): u* gains J / (Z_L + Z_R) and the two
                                    sides of a face see p* -/+ J/2, J = sigma kappa_f
                                    (alpha_i+1 - alpha_i) with kappa_f the mean of the cells'
                                    curvatures (the curvature option above).  The jump model
                                    runs the tiled stage kernel and is not combined with
                                    viscous terms, slabs of a split grid or the no-alloc stage
                                    (FV_ERR_ARG). */
} fv_eos;

typedef struct fv_ctx fv_ctx;

/* Bytes of device workspace fv_init_ws needs for these cases. */
fv_status fv_workspace_size(int ncases, const fv_grid* grids, const fv_components* comps,
                            const fv_eos* eos, size_t* bytes);

/* Create a context for ncases independent cases sharing components and
 * scheme (ncases = 1: a single grid).  fv_init allocates device memory with
 * cudaMalloc; fv_init_ws uses the caller's device buffer of at least
 * fv_workspace_size bytes (256-byte aligned), which must outlive the context.
 * The context uses the current CUDA device and the legacy default stream
 * until fv_set_stream.  Errors: FV_ERR_ARG (bad sizes, unsupported closure or
 * boundary mix), FV_ERR_ALLOC, FV_ERR_CUDA.  On an error *out may still hold
 * a context whose fv_last_error explains it; release it with fv_destroy. */
fv_status fv_init(int ncases, const fv_grid* grids, const fv_components* comps, const fv_eos* eos,
                  fv_ctx** out);
fv_status fv_init_ws(int ncases, const fv_grid* grids, const fv_components* comps, const fv_eos* eos,
                     void* dev_workspace, size_t bytes, fv_ctx** out);
void fv_destroy(fv_ctx* ctx);

/* One grid split into nblocks slabs along its last dimension (y in 2D, z in
 * 3D), the decomposition that distributes a grid over several GPUs: the
 * compact stencil of Sec. 3.1 needs two ghost layers, so before every stage
 * each slab receives the two planes of the stage's input state next to each
 * side it shares with a neighbouring slab (device-to-device copies), and
 * every step takes the smallest dt of all slabs.  The slabs are the
 * context's cases: case b holds planes row0_b .. row0_b + rows[b] - 1 of the
 * split dimension, and the per-case calls (fv_set_state, fv_get_state, ...)
 * address one slab with that slab's part of the layout above.  rows (may be
 * NULL: as even as possible) gives each slab's plane count, each at least 2,
 * summing to the grid's extent; a periodic split dimension joins the last
 * slab to the first.  The result equals the unsplit grid's, bit for bit.
 * dev_workspace NULL: cudaMalloc; otherwise at least fv_split_workspace_size
 * bytes (256-byte aligned).  Errors as for fv_init. */
fv_status fv_split_workspace_size(const fv_grid* grid, int nblocks, const int* rows, const fv_components* comps,
                                  const fv_eos* eos, size_t* bytes);
fv_status fv_init_split(const fv_grid* grid, int nblocks, const int* rows, const fv_components* comps,
                        const fv_eos* eos, void* dev_workspace, size_t bytes, fv_ctx** out);

/* Stream (a cudaStream_t) for all later work of the context. */
fv_status fv_set_stream(fv_ctx* ctx, void* stream);

/* Copy a case's state from/to host memory (kind FV_CONSERVED or
 * FV_PRIMITIVE; nv * n[0]*n[1]*n[2] doubles).  Primitive input is turned
 * into conserved variables by the closure on the device.  Page-locked host
 * memory (cudaHostAlloc / cudaHostRegister) is read or written by the
 * device's conversion kernel directly over the host link; other host memory
 * is staged through a device buffer.  Synchronous: returns once the copy is
 * complete.  get_state also reports a pending device error word as
 * FV_ERR_NONPHYSICAL / FV_ERR_EOS_NONCONV. */
fv_status fv_set_state(fv_ctx* ctx, int icase, int kind, const double* host);
fv_status fv_get_state(fv_ctx* ctx, int icase, int kind, double* host);
/* Every case in one call, for batches of many small cases: `host` holds
 * each case's block of the layout above (nv * cells doubles) concatenated in
 * case order.  Conserved state in page-locked host memory is moved by one
 * kernel over all cases; other memory, and primitive input, goes case by
 * case.  One synchronisation per call; errors as for fv_set_state /
 * fv_get_state. */
fv_status fv_set_state_all(fv_ctx* ctx, int kind, const double* host);
fv_status fv_get_state_all(fv_ctx* ctx, int kind, double* host);
/* Pipelined conserved-state I/O of every case (the layout of
 * fv_set_state_all), for a stream of problems whose host transfers should
 * overlap the steps: the copies run on the device's copy engines through
 * device staging buffers, two each way used in turn so that consecutive
 * copies follow one another without waiting for the conversions (allocated
 * with cudaMalloc at the first call: four times the state's size; freed by
 * fv_destroy), uploads and downloads on two streams of their own.
 *   fv_upload_async   starts copying `host` (page-locked) to the next upload
 *                     staging buffer; returns at once.  One upload may be
 *                     pending: FV_ERR_STATE if the previous one is not yet
 *                     committed.
 *   fv_commit_upload  makes the context's stream wait for that copy and
 *                     turns it into the current state (the case clocks
 *                     restart); the next fv_upload_async may then start.
 *   fv_download_async queues, on the context's stream after the work already
 *                     queued, a copy of the current state to `host`
 *                     (page-locked), which must stay untouched until
 *                     fv_io_wait returns.
 *   fv_io_wait        waits for every transfer and the context's stream and
 *                     reports a pending device error word.
 * A host buffer passed to fv_upload_async may be reused once the matching
 * fv_commit_upload's work has run (fv_io_wait, or a later download that
 * completed). */
fv_status fv_upload_async(fv_ctx* ctx, const double* host);
fv_status fv_commit_upload(fv_ctx* ctx);
fv_status fv_download_async(fv_ctx* ctx, double* host);
fv_status fv_io_wait(fv_ctx* ctx);

/* Same with device pointers; asynchronous on the context's stream. */
fv_status fv_set_state_device(fv_ctx* ctx, int icase, int kind, const double* dev);
fv_status fv_get_state_device(fv_ctx* ctx, int icase, int kind, double* dev);

/* One Runge-Kutta stage k = 1..4 of every case with a caller-given dt
 * (q^k = q^0 + a_k dt R(q^{k-1}); stage 1 starts from the current state,
 * stage 4 writes the new state).  Stages must be called in order. */
fv_status fv_rk_stage(fv_ctx* ctx, int k, double dt);

/* The first fv_rk_stage / fv_step of a context autotunes the stage kernel on
 * the current state (a few timed launches per candidate that write only a
 * scratch register; cached per workload class for the process).  Candidates:
 * the tiled kernel's tile shapes (each after a primitive pass) and, for 2D
 * grids in plain mode with the stiffened/ideal-gas closure, a fused kernel
 * that recovers the primitives itself (one pass per stage, no primitive
 * pass), and for 3D grids in the FP32-mixed form with the stiffened/ideal-gas
 * closure a kernel that marches along z with TMA plane loads.
 * FV_TILE=<index> in the environment forces a tile of the tiled kernel,
 * FV_FUSED=0/1 and FV_ZMARCH=0/1 exclude or force the fused and the
 * z-marching kernel, FV_ZVAR=<v> keeps only the z-marching kernel's variant
 * v (0/1/3/4/5: 320/256/352/416/288 threads with the Table 4.2 limiter
 * pair; 2: run-time limiter pair; the viscous form has 1 and 2, the FP64
 * form 1, 2, 4 and 5), FV_FUSED_CFL=0 (read when the context is created)
 * keeps the CFL pass in every step of the fused kernel (see fv_step).  Set
 * the state first. */

/* nsteps full steps: per step dt = cfl / max(sum_d (|u_d| + c)/dx_d) of each
 * case, with viscous terms plus 2 D sum_d 1/dx_d^2 under the maximum,
 * D = max(4/3 mu, k_c / cv_min)/rho and cv_min the smallest component cv
 * (the paper defines no step: both are readings), computed on the device
 * from the step's initial state; then the four stages.  The step sequence is captured once per cfl value in a CUDA graph
 * and replayed on the context's stream.  With the fused 2D kernel in the
 * FP32-mixed form (no viscous or gravity terms) the last stage of a step
 * also leaves the wave speeds of the state it writes, and the next step
 * (within this call or the next fv_step / fv_step_async) takes its dt from
 * them instead of a CFL pass over the state; a state write in between
 * (fv_set_state*, fv_commit_upload, fv_rk_stage) makes the next step
 * compute them again.  Both give the same dt bit for bit.  t_out (may be
 * NULL) receives case 0's simulated time since its last fv_set_state.
 * Synchronises the stream once at the end and reports a device error word
 * (FV_ERR_NONPHYSICAL). */
fv_status fv_step(fv_ctx* ctx, int nsteps, double cfl, double* t_out);
/* Same without any host synchronisation or readback (for timing loops). */
fv_status fv_step_async(fv_ctx* ctx, int nsteps, double cfl);

/* Diagnostics of one case (see FV_DIAG_*); synchronous. */
fv_status fv_get_diag(fv_ctx* ctx, int icase, int what, void* out);

/* Counters of kernel launches issued so far (for launch accounting). */
long long fv_launch_count(const fv_ctx* ctx);

/* Kernel timing: with enable = 1, fv_step / fv_step_async / fv_rk_stage
 * launch the kernels directly (no graph) and record a CUDA event pair on the
 * context's stream around every launch; enable = 0 stops recording and frees
 * the events.  fv_profile_read synchronises and returns, per kernel kind
 * (FV_KERNEL_*), out[2*kind] = total milliseconds and out[2*kind+1] = number
 * of launches since recording started. */
enum { FV_KERNEL_PRIM = 0, FV_KERNEL_DT = 1, FV_KERNEL_STAGE = 2, FV_KERNEL_KINDS = 3 };
fv_status fv_profile(fv_ctx* ctx, int enable);
fv_status fv_profile_read(fv_ctx* ctx, double* out);

const char* fv_last_error(const fv_ctx* ctx);
const char* fv_status_string(int status);

/* Self-test of the kernels' bounded waits (the TMA tile and plane copies
 * wait on an mbarrier with a poll limit): one block waits `polls` polls on an
 * mbarrier that nothing completes and takes the give-up path.  *err_word
 * receives the device error word (FV_ERRBIT_TIMEOUT expected); the device
 * stays usable.  Synchronous, on the legacy default stream; not a paper
 * operation. */
fv_status fv_wait_selftest(int polls, int* err_word);

/* FP64 arithmetic-rate probe for the FP64 form's roofline (not a paper
 * operation): blocks x threads threads each run `iters` rounds of eight
 * independent FP64 fused multiply-adds; *ms receives the CUDA-event time of
 * one launch (after a warm-up launch) and *flops the flops it performed
 * (2 per FMA).  Synchronous, on the legacy default stream. */
fv_status fv_probe_fp64(int blocks, int threads, int iters, double* ms, double* flops);

/* One Runge-Kutta stage of one grid that allocates no device memory, for
 * callers that cannot call cudaMalloc: code that runs inside a host
 * application owning the whole device through its own memory pool, code
 * with a fixed memory budget set before it starts, or code on a path where
 * an allocation (and the synchronisation it can imply) is not allowed.  The
 * paper has no counterpart; it is the fv_rk_stage arithmetic on the same
 * kernels with the scratch held in a static device array of
 * FV_NOALLOC_SCRATCH_BYTES per GPU, kept from library load until exit.
 *
 * q0 (the step's initial state), qprev (stage k-1's output; q0 for k = 1) and
 * qout are caller-owned device arrays in the conserved layout above; qout
 * receives q0 + a_k dt R(qprev).  qout may be q0 itself (as stage 4 does) but
 * may not overlap qprev or part of q0 (FV_ERR_ARG).  Limit: the primitive
 * scratch of (n+4)^d ghosted cells times (ndim + ncomp + 1 + extra fields)
 * values of 8 bytes (FV_FP64) or 4 bytes (FV_MIXED), plus small work lists,
 * must fit the array; larger grids, a per-cell inflow array (grid->in_u), the
 * barotropic closure in the FV_MIXED form, Peng-Robinson components, the
 * capillary-jump surface-tension model (st_model = 1 with sigma > 0) and
 * every argument fv_init would reject return FV_ERR_ARG.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) with that device
 * current and keeps it for the process; do not reset the device
 * (cudaDeviceReset) after it.
 * Every call uses the same array: calls that overlap on the GPU (other
 * streams, other threads) race.  The call runs on `stream` and returns once
 * the stage has finished, reporting a non-physical state met by the kernels
 * as FV_ERR_NONPHYSICAL and a kernel wait that gave up as FV_ERR_CUDA. */
#define FV_NOALLOC_SCRATCH_BYTES (48u << 20)
fv_status fv_rk_stage_noalloc(const fv_grid* grid, const fv_components* comps, const fv_eos* eos,
                              int k, double dt, const double* q0, const double* qprev, double* qout,
                              void* stream);

#ifdef __cplusplus
}
#endif
#endif
