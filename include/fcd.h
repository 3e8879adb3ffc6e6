/*
 * fcd.h -- C ABI of the GB300 (sm_103a) coupled time step of the ferrofluid
 * compound-droplet model of arXiv 2410.11129 ("Deformation and breakup of a
 * ferrofluid compound droplet migrating in a microchannel under a magnetic
 * field: a phase-field-based multiple-relaxation time lattice Boltzmann study").
 *
 * One step advances, on one GPU:
 *   - the phase fields phi_1 (core), phi_2 (shell) by the conservative
 *     Allen-Cahn lattice Boltzmann equation (Sec. 2.3-2.4, Eqs. 23-32),
 *   - the magnetic scalar potential psi of div[(1+chi) grad psi] = 0 under a
 *     uniform field H0 at angle alpha (Sec. 2.1, Eqs. 1-9), solved by multigrid,
 *   - the ternary flow by the D2Q9 MRT lattice Boltzmann equation with surface
 *     tension, Kelvin, pressure, viscous and driving forces (Sec. 2.2, Eqs. 10-22),
 *   - half-way bounce-back walls at y = -1/2 and y = ny - 1/2, periodic x.
 *
 * Conventions shared by every call:
 *   - Every call returns an fcd_status; none aborts, traps or exits. On failure
 *     fcd_last_error() holds a one-line reason.
 *   - The context owns its device memory (allocated in fcd_create through the
 *     allocator installed by fcd_set_allocator, else cudaMalloc) and frees it in
 *     fcd_destroy. Buffers passed in by the caller stay the caller's.
 *   - Work is queued on the context's stream (fcd_set_stream; default: the
 *     legacy default stream). fcd_step returns once the work is queued; calls
 *     that return data to the host synchronise that stream.
 *   - Lattice units: dx = dt = 1, c_s^2 = 1/3, mu0 = 1.
 *   - Field arrays exchanged with the caller are FP64, row-major, unpadded:
 *     a[y*nx + x]; populations f[a][y][x] (9 planes, D2Q9 order rest, E, N,
 *     W, S, NE, NW, SW, SE), g[i][a][y][x] (2 x 9 planes, i = 0 core, 1 shell).
 *     Pointers may be host or device memory (unified addressing decides).
 */
#ifndef FCD_H
#define FCD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fcd_ctx fcd_ctx;

typedef enum {
    FCD_OK = 0,
    FCD_EINVAL = 1,     /* bad argument or parameter set */
    FCD_ENOMEM = 2,     /* device allocation failed */
    FCD_ECUDA = 3,      /* a CUDA call failed; the message names it */
    FCD_ENOCONV = 4,    /* potential solve hit its cycle cap before the tolerance */
    FCD_EUNSTABLE = 5,  /* non-finite values detected: a collision that produced a
                         * non-finite velocity or pressure marks its step on the
                         * device (no trap; the steps complete) and the next
                         * fcd_observables, fcd_get_field or fcd_get_populations
                         * returns this status with that step in fcd_last_error;
                         * fcd_observables also flags a non-finite phase field.
                         * fcd_set_populations and fcd_set_state clear the record. */
    FCD_ESTATE = 6      /* snapshot does not match this context */
} fcd_status;

/* Storage forms of the populations. FP64; FP32 storing f + w_a and g as they
 * are; FP32 "offset" storing f (an offset from the weights in this
 * velocity-based form) and g - w_a/2, with each node's rest population g_0 set
 * to the exact remainder of its pre-collision sum, rounded to FP32 without
 * bias (reproducibly, from a hash of node, step and phase), so that the phase
 * masses only random-walk by one rounding per node and step. FP32 contexts
 * created with mag_tol below 1e-4 also hold psi' as a hi + lo pair. */
typedef enum { FCD_FP64 = 0, FCD_FP32 = 1, FCD_FP32_OFFSET = 2 } fcd_precision;

/* Problem statement of Sec. 2.5 in lattice units. Phases: 1 core, 2 shell,
 * 3 carrier (index 0, 1, 2 in the arrays). */
typedef struct {
    int nx, ny;            /* lattice nodes along / across the channel; nx even, >= 4; ny >= 2 */
    double rho[3];         /* densities (Eq. 33 mixes them linearly) */
    double nu[3];          /* kinematic viscosities; tau_i = nu_i / c_s^2 (Eq. 14) */
    double chi[3];         /* magnetic susceptibilities (Eq. 8 mixes 1 + chi harmonically) */
    double mobility;       /* M of Eq. 30 (0.3 in the paper) */
    double xi;             /* interface width (Eq. 23; 5 in the paper) */
    double eta;            /* Eq. 28 eta (0: partial spreading) */
    double Ca;             /* Eq. 40, fixes sigma_23 = rho3 nu3 u_avg / Ca */
    double Bo_m;           /* Eq. 41, fixes mu0 H0^2 */
    double alpha;          /* field angle to the x axis, radians */
    double r1, r2;         /* core and shell radii */
    double xc, yc;         /* droplet centre */
    double s13_over_s12;   /* sigma_13 / sigma_12 (Table 2) */
    double s23_over_s12;   /* sigma_23 / sigma_12 (Table 2) */
    double sigma23;        /* > 0: use this sigma_23 instead of the Eq. 40 relation */
    double u_max;          /* centre-line speed of the body-force-driven channel flow */
    int ferro_phase;       /* 1 core, 2 shell, 0 none: selects the Eq. 41 branch */
    int precision;         /* fcd_precision: storage and arithmetic of the populations */
    double mag_tol;        /* potential solve target ||L psi||_inf / H0 per step */
    int mag_max_iter;      /* multigrid V-cycle cap per solve */
    double eps_n;          /* regulariser of n = grad phi / (|grad phi| + eps_n) */
    int open_x;            /* 0: periodic channel driven by a body force (u_max).
                            * 1: the paper's open channel (Sec. 2.5): the Eq. 37
                            * parabola (centre-line speed u_max) enters at x = 0 as
                            * pure carrier, a convective outlet at x = nx - 1 holds
                            * the reference p* = 0; no body force. The potential
                            * psi' stays periodic in x. */
} fcd_params;

/* Observables (Sec. 2.5, Eqs. 38 and 42). */
typedef struct {
    long step;              /* time steps taken since fcd_create */
    double t_star;          /* Eq. 38: step * u_avg / (2 r2), u_avg = 2 u_max / 3 */
    double T_o, T_i;        /* Eq. 42 deformation of the shell and the core */
    double lx_o, ly_o, lx_i, ly_i; /* extents of the 1/2 level sets */
    double xc_core, yc_core, xc_shell, yc_shell; /* indicator-weighted centroids */
    double mass[3];         /* sum over nodes of phi_1, phi_2, phi_3 (FP64) */
    int breakup;            /* 1 once the core has touched the carrier */
    long b_step;            /* step of the first touch, -1 if none */
    double xb, yb;          /* node of the first touch (smallest (y, x)) */
    double tb_star, Lb_star, yb_star; /* t_b* (Eq. 38), x_b / H, |y_b - centre| / H */
    int mag_iters;          /* V-cycles of the most recent potential solve */
    double mag_resid;       /* its final ||L psi||_inf / H0 */
} fcd_obs;

/* Fields for fcd_get_field (FP64, nx*ny values). The macroscopic fields are
 * those of the most recent collision (initial values right after create). */
typedef enum {
    FCD_FIELD_PHI1 = 0, FCD_FIELD_PHI2 = 1, FCD_FIELD_PHI3 = 2,
    FCD_FIELD_UX = 3, FCD_FIELD_UY = 4, FCD_FIELD_PSTAR = 5, FCD_FIELD_PSI = 6
} fcd_field;

/* Optional allocator used by later fcd_create calls (process-wide; NULL
 * restores cudaMalloc/cudaFree). alloc returns a device pointer or NULL. */
typedef void *(*fcd_alloc_fn)(size_t bytes, void *user);
typedef void (*fcd_free_fn)(void *ptr, void *user);
void fcd_set_allocator(fcd_alloc_fn alloc, fcd_free_fn release, void *user);

/* Maps the dimensionless groups to lattice units (Eqs. 14, 26-27, 30, 40-41),
 * allocates the state, sets the initial condition (concentric tanh profiles
 * of width xi, Poiseuille flow, f = f^eq, g = phi Gamma) and solves the
 * potential once. EINVAL for nx odd or < 4, ny < 2, r1 > r2, non-positive
 * density, viscosity, mobility or xi, eta < 0, a gamma_i = 0 (Eq. 26
 * undefined), total spreading (a gamma_i < 0, Eq. 27) with eta = 0 (Eq. 28
 * needs eta > 0 then), gamma_1 gamma_2 + gamma_1 gamma_3 + gamma_2 gamma_3 <= 0
 * (gradient energy not positive), or an Eq. 41 branch without a magnetic
 * phase. *out is NULL on failure. */
fcd_status fcd_create(const fcd_params *params, fcd_ctx **out);

/* Queue later work on this cudaStream_t (passed as void*). */
fcd_status fcd_set_stream(fcd_ctx *ctx, void *cuda_stream);

/* Advance n >= 0 coupled steps: phase recovery (Eq. 32), permeability (Eq. 8),
 * potential solve (Eq. 6, to mag_tol or mag_max_iter V-cycles), forces and
 * velocity (Eqs. 5-9, 19-22, 25-28, 33-36), MRT collision of f (Eqs. 12-18),
 * BGK collision of g^1, g^2 (Eqs. 29-31), push streaming with bounce-back.
 * Asynchronous; an unconverged solve is reported by the next synchronising
 * call as FCD_ENOCONV. */
fcd_status fcd_step(fcd_ctx *ctx, long n);

/* Solve the potential for the current phase fields (Eqs. 6-8). Synchronous.
 * tol <= 0 or max_iter <= 0 take the values from the parameters. */
fcd_status fcd_solve_magnetic(fcd_ctx *ctx, double tol, int max_iter, int *iters,
                              double *resid);

/* Observables of the current state (Eqs. 38, 42; breakup of Sec. 2.5). Synchronous. */
fcd_status fcd_observables(fcd_ctx *ctx, fcd_obs *out);

/* Copy one field (fcd_field) into dst (nx*ny doubles, host or device). Synchronous. */
fcd_status fcd_get_field(fcd_ctx *ctx, int which, double *dst, size_t n);

/* Populations and perturbation potential psi' in the FP64 exchange layout
 * (f: 9*nx*ny, g: 18*nx*ny, psi: nx*ny); any pointer may be NULL to skip it.
 * set_populations also sets the step counter and clears the breakup record. */
fcd_status fcd_get_populations(fcd_ctx *ctx, double *f, double *g, double *psi);
fcd_status fcd_set_populations(fcd_ctx *ctx, const double *f, const double *g,
                               const double *psi, long step);

/* Opaque snapshot (stored populations in the context's precision, psi',
 * step, breakup record) for checkpoint and resume; resuming reproduces an
 * uninterrupted run bit for bit. */
size_t fcd_state_bytes(const fcd_ctx *ctx);
fcd_status fcd_get_state(fcd_ctx *ctx, void *dst, size_t bytes);
fcd_status fcd_set_state(fcd_ctx *ctx, const void *src, size_t bytes);

/* Derived lattice quantities (Eqs. 14, 26-27, 30, 40-41): [u_avg, sigma12,
 * sigma13, sigma23, gamma1..3, gammaT, tau1..3, tau_phi, mu0H0^2, H0, G]
 * (15 doubles). */
fcd_status fcd_get_derived(const fcd_ctx *ctx, double *out15);

/* The same 15 derived quantities straight from a parameter set, without a
 * context: the lattice mapping of Sec. 2.5 (Eq. 40: sigma23 from Ca; Eq. 41:
 * mu0 H0^2 from Bo_m, core or shell branch; Eqs. 14, 26-27, 30). Host code
 * only: no CUDA call, no allocation. FCD_EINVAL (reason in fcd_last_error(NULL))
 * for a parameter set that fcd_create would reject. */
fcd_status fcd_derive_params(const fcd_params *params, double *out15);

/* Number of kernels launched by this context since create (for accounting;
 * synchronises to read the device-side cycle count). */
long fcd_kernel_launches(const fcd_ctx *ctx);

/* Cumulative potential-solver counters since create: [cycle heads (lattice
 * residual evaluations), V-cycles, two-grid cycles, lattice-sweep cycles,
 * solves stopped at the cycle cap] (synchronises). */
fcd_status fcd_solver_stats(fcd_ctx *ctx, long long *out5);

/* Rows per tile of the fused collide-stream kernel (Sec. 2.2-2.4 update,
 * 32 nodes wide). FP32 contexts time 4 and 8 rows at create on their own grid
 * and keep the faster (both do the same arithmetic per node, so the results do
 * not depend on the choice); the environment variable FCD_COLLIDE_TILE_H=4 or 8,
 * set before create, fixes it. FP64 and tangent contexts use 8 and 4.
 * FCD_EINVAL for a null argument. */
fcd_status fcd_collide_tile_height(const fcd_ctx *ctx, int *rows);

/* Timing of the stages of a step with CUDA events recorded on the context's
 * stream (inside the step graph): enable, run fcd_step, then read
 * ms4 = [phase recovery + coarse permeabilities, potential solve,
 * collide-stream, whole step] of the most recent step (synchronises). */
fcd_status fcd_set_profiling(fcd_ctx *ctx, int enable);
fcd_status fcd_last_step_profile(fcd_ctx *ctx, double *ms4);

/* Reason of the last failure on ctx; with ctx == NULL, of the last failed
 * fcd_create on the calling thread. */
const char *fcd_last_error(const fcd_ctx *ctx);

/* ---- Batched form: many independent channels (the Bo_m x Ca regime map of
 * Sec. 3.7 is a grid of separate runs). Each instance is a full context (its
 * own state; every fcd_* call works on it). Two ways to step them (see
 * fcd_batch_tuning): the periodic FP32 instances of one storage form and one
 * level-0 form of the potential (a tolerance below 1e-4 or not) advanced
 * together by one fixed set of kernels per step, each launched once over a
 * work list of tiles that spans them (phase recovery, a single loop of
 * batched multigrid kernels in which every instance runs the cycle its own
 * residual chose, and the fused collide-stream, whose tile height an
 * autotuner picks at create by timing), the other instances (FP64, open
 * channels) on their own streams beside them; or every instance's own step
 * graph on its own stream. The first steps time both and keep the faster.
 * fcd_batch_step then makes the caller's stream wait for everything.
 * On their own streams (mode 0 of fcd_batch_tuning) the instances' results
 * are bit-identical to stepping each alone; the batched kernels agree with
 * them to the rounding of contracted multiply-adds. */
typedef struct fcd_batch fcd_batch;
/* n parameter sets (instances may differ in every field, sizes included). */
fcd_status fcd_batch_create(const fcd_params *params, int n, fcd_batch **out);
/* Stream that fcd_batch_step orders itself after and joins into (default: legacy stream). */
fcd_status fcd_batch_set_stream(fcd_batch *b, void *cuda_stream);
/* Advance every instance by n steps (asynchronous, like fcd_step). */
fcd_status fcd_batch_step(fcd_batch *b, long n);
/* Observables of every instance into out[0..size-1] (synchronous); the first
 * non-OK instance status is returned. */
fcd_status fcd_batch_observables(fcd_batch *b, fcd_obs *out);
int fcd_batch_size(const fcd_batch *b);
/* How the batch steps. *mode: 1 = the batched kernels for the groups, 0 =
 * every instance's own step graph on its own stream, all at once (the results
 * of the two agree to the rounding of the fused multiply-adds the compiler
 * forms in each kernel variant); -1 while the first steps still time both: 6
 * single steps, the first two of which build the graphs, the last four timed
 * alternately; the faster mode is kept (the environment variable
 * FCD_BATCH_MODE=0 or 1 at create fixes it instead). *batched = instances the
 * batched kernels advance, *groups = their groups (each set of one storage
 * form and one level-0 potential form split
 * into about one group per 6 M lattice nodes, at most 8, balanced by nodes,
 * each group on its own stream; FCD_BATCH_GROUPS=k at create fixes the
 * split), tile_h[g] for g < tile_h_len = the collide-stream tile height the
 * autotuner chose for group g at create. Any pointer may be NULL. An instance
 * stepped on its own (fcd_step) leaves its group out of phase with it; that
 * group then steps its instances one by one until their parities agree again. */
fcd_status fcd_batch_tuning(const fcd_batch *b, int *mode, int *batched, int *groups, int *tile_h,
                            int tile_h_len);
/* Fix the stepping mode (0 or 1, as above) or time both again (-1). EINVAL for
 * mode 1 when no instance can take the batched kernels. */
fcd_status fcd_batch_set_mode(fcd_batch *b, int mode);
/* Instance i (owned by the batch; use any fcd_* call on it, not fcd_destroy). */
fcd_ctx *fcd_batch_instance(fcd_batch *b, int i);
/* Reason of the last failure on b; with b == NULL, of the last failed create. */
const char *fcd_batch_last_error(const fcd_batch *b);
void fcd_batch_destroy(fcd_batch *b);

/* ---- Tangent-linear form: exact discrete derivatives of the coupled step
 * (forward mode) with respect to the four parameters of the regime study,
 * direction order FCD_DIR_BO_M (Bo_m, Eq. 41), FCD_DIR_CA (Ca, Eq. 40),
 * FCD_DIR_ALPHA (alpha, radians), FCD_DIR_NU_R (nu_r = nu_3 / nu_2, Eq. 39).
 * A tangent context is an FP64 context (precision is ignored) whose state also
 * carries the derivative of every population, phase field and potential along
 * the four directions; each step applies the chain rule to the whole step:
 * the collision and streaming in dual arithmetic, and four extra potential
 * solves L(k) dpsi' = b(k, dH0) + b(dk, H0) - L(dk) psi' with the same
 * multigrid (differentiating Eq. 6 with psi = psi0 + psi'), each to
 * mag_tol relative to the largest |right-hand side|. Bo_m must be > 0 when a
 * phase is ferrofluid (H0 ~ sqrt(Bo_m)); with sigma23 > 0 given directly the
 * Ca direction is zero. The returned handle accepts fcd_step, fcd_observables
 * (primal values), fcd_get_field (primal fields), fcd_kernel_launches,
 * fcd_solver_stats, fcd_last_error and fcd_destroy; state snapshots and
 * population import return FCD_ESTATE. Each step runs as one captured CUDA
 * graph (the primal and the four tangent solves as conditional-node loops, as in
 * fcd_step), with no host synchronisation between steps; with the environment
 * variable FCD_NO_GRAPH=1 the solves are driven from the host instead, one
 * synchronisation per multigrid cycle. */
enum { FCD_DIR_BO_M = 0, FCD_DIR_CA = 1, FCD_DIR_ALPHA = 2, FCD_DIR_NU_R = 3, FCD_NDIR = 4 };
typedef struct {
    long step;
    double T_o;                 /* shell deformation (Eq. 42), same value as fcd_observables */
    double overlap;             /* sum over nodes of phi_1 phi_3 (core-carrier overlap, unclamped) */
    double lx_o, ly_o;          /* shell extents along and across the channel */
    double dT_o[FCD_NDIR];      /* dT_o / d(Bo_m, Ca, alpha, nu_r) */
    double doverlap[FCD_NDIR];  /* d overlap / d(...) */
    double dlx_o[FCD_NDIR], dly_o[FCD_NDIR];
} fcd_tangent_obs;
fcd_status fcd_create_tangent(const fcd_params *params, fcd_ctx **out);
/* Values and derivatives of the current state (synchronous). T_o is
 * differentiated through the crossing interpolation of the 1/2 level set
 * (l_x: the two centre-line crossings; l_y: the column of largest extent). */
fcd_status fcd_tangent_observables(fcd_ctx *ctx, fcd_tangent_obs *out);

/* ---- Discrete adjoint (reverse mode): gradients of one scalar functional of
 * the final state, J = w_T T_o + w_overlap sum_nodes phi_1 phi_3 (T_o of
 * Eq. 42; the overlap as in fcd_tangent_obs), with respect to the four
 * parameters of the tangent form (same direction order) and to the initial
 * populations. An adjoint context is an FP64 channel, periodic or open
 * (precision is ignored), that keeps a checkpoint of its state every
 * checkpoint_interval steps from step 0 (device memory: 30 planes of nx*ny
 * doubles per checkpoint). fcd_adjoint_gradient runs the reverse sweep from the
 * current step N back to step 0, one segment between checkpoints at a time,
 * last first: the segment's forward states are recomputed from its checkpoint
 * into checkpoint_interval slots (28 planes each, allocated by the first step;
 * FCD_ENOMEM if they do not fit), then the adjoint of every step runs backwards
 * through them. fcd_step keeps the states of the current segment in the slots,
 * so the last segment is not recomputed (none is when checkpoint_interval >= N).
 * Each adjoint step reverses the open channel's boundary populations (inlet of
 * Eq. 37, convective outlet) when open_x = 1, the collision and streaming of
 * every node, and the potential solve: L(k) lam = psib (L of Eq. 6 is
 * symmetric) with the multigrid of the plain solve to mag_tol relative to
 * max |psib|, then the permeability and field-strength adjoints of
 * b(k, H0) - L(k) psi'. Bo_m must
 * be > 0 when a phase is ferrofluid. The handle accepts fcd_step (forward, with
 * checkpoints), fcd_observables, fcd_get_field, fcd_solve_magnetic,
 * fcd_kernel_launches, fcd_solver_stats, fcd_last_error and fcd_destroy; state
 * snapshots and population import return FCD_ESTATE (they would cut the
 * recorded trajectory). checkpoint_interval >= 1, else FCD_EINVAL. */
typedef struct {
    long step;                  /* N, the step of the final state */
    double T_o, overlap;        /* values at step N */
    double J;                   /* w_T T_o + w_overlap overlap */
    double grad[FCD_NDIR];      /* dJ / d(Bo_m, Ca, alpha, nu_r) */
    long capped_solves;         /* adjoint potential solves that stopped at mag_max_iter */
    long recomputed_steps;      /* forward steps the sweep recomputed from checkpoints */
    long long solve_cycles;     /* multigrid cycles of the sweep's adjoint potential solves */
} fcd_adjoint_out;
fcd_status fcd_create_adjoint(const fcd_params *params, int checkpoint_interval, fcd_ctx **out);
/* Reverse sweep (synchronous). df0, dg0: NULL, or host or device buffers of
 * 9*nx*ny and 18*nx*ny doubles (layout of fcd_get_populations) that receive
 * dJ / d(f, g at step 0). The context is back at step N afterwards, also when
 * the sweep fails. Returns FCD_ENOCONV (with out filled) when an adjoint solve
 * stopped at the cap. With w_T = w_overlap = 0 and no df0, dg0 the call only
 * fills the values (J = 0 has a zero gradient; no sweep runs). */
fcd_status fcd_adjoint_gradient(fcd_ctx *ctx, double w_T, double w_overlap, fcd_adjoint_out *out,
                                double *df0, double *dg0);
/* The same sweep for any functional J of the final state, given by its
 * derivative: seed_f, seed_g = dJ/d(f, g at step N) in the layout of
 * fcd_get_populations (9*nx*ny and 18*nx*ny doubles, host or device memory;
 * one of them may be NULL, meaning zero; both NULL is FCD_EINVAL). out->grad
 * and df0, dg0 as above; out->T_o and out->overlap are the state's values and
 * out->J is 0 (J is the caller's). Synchronous; the context stays at step N. */
fcd_status fcd_adjoint_gradient_state(fcd_ctx *ctx, const double *seed_f, const double *seed_g,
                                      fcd_adjoint_out *out, double *df0, double *dg0);

/* Observables of a caller's population buffer with no device allocation.
 * The paper has no counterpart: this serves callers that cannot allocate
 * device memory (another framework owns the memory budget, cudaMalloc/cudaFree
 * would synchronise a latency-critical loop, or the memory plan is fixed in
 * advance). g: device pointer to the phase-field populations in the FP64
 * exchange layout (18*nx*ny doubles, g[i][a][y][x]); nx >= 4, ny >= 2,
 * nx <= 16384 and nx*ny <= 524288, else FCD_EINVAL with the reason on stderr.
 * open_x: 0 for the periodic channel, 1 for the open channel (fcd_params.open_x;
 * the extents and the breakup neighbourhood then do not wrap in x), as the
 * context that produced the state. Fills mass, centroids, extents, T_o, T_i
 * and the breakup fields of the given state (b_step = 0 if the core touches
 * the carrier in it, else -1); step, t_star and the solver fields are 0. Work
 * runs on cuda_stream (a cudaStream_t; NULL = legacy default stream) and the
 * call synchronises it.
 * Scratch: one 9.5 MiB device array inside the library, reserved on every
 * GPU that loads it until the process exits; its device address is looked up
 * (cudaGetSymbolAddress) by the first call on each device and kept, so make
 * that first call before any stream capture; after cudaDeviceReset (or any
 * teardown of the device's primary context) the kept address is stale and
 * this entry point must not be called again in the process. All calls share
 * that array: calls that may overlap on the GPU (other streams, other host
 * threads) race and must be serialised by the caller. Allocates nothing: no
 * cudaMalloc, cudaFree or allocating library routine. */
fcd_status fcd_observe_populations_noalloc(const double *g, int nx, int ny, int open_x,
                                           void *cuda_stream, fcd_obs *out);
void fcd_destroy(fcd_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif
