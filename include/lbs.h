/*
 * lbs.h — C ABI of the GB300 hybrid lattice Boltzmann / finite-difference
 * solver for two-phase flow with soluble surfactants (Ba, Liu, Li & Yang,
 * arXiv 2311.15242).
 *
 * One call of lbs_step advances the coupled update of the paper by one time
 * step on the GPU, on a D2Q9 (nz == 1) or D3Q19 (nz > 1) lattice:
 *   Sec. 2.1   colour-gradient LB step: MRT collision with the correction
 *              term and the forcing term (Eqs. 1-4, App. A Eqs. 36-43: D2Q9
 *              Eqs. 36-38, D3Q19 Eqs. 39-41), the
 *              interfacial force from the modified Langmuir equation of state
 *              with the Marangoni term (Eqs. 5-9), the velocity of Eq. 10,
 *              recolouring (Eqs. 11-12), streaming with half-way bounce-back
 *              (Eq. 13);
 *   Sec. 2.2   finite-difference update of the interface and bulk surfactant
 *              equations (Eqs. 20-22): WENO3 convection (Eqs. 25-27),
 *              Crank-Nicolson diffusion (Eqs. 23-24, 28) solved by red-black
 *              SOR with omega = 1.2, rescaling of the total surfactant.
 *
 * Conventions (all entry points):
 *   - every function returns an lbs_status (0 = success) unless noted; no
 *     exception or abort crosses the ABI; lbs_last_error() describes the
 *     last failure of a context;
 *   - host arrays are caller-owned, double precision, row-major [z][y][x]
 *     (x fastest) with N = nx*ny*nz entries per scalar field and 3*N for a
 *     vector field (component-major: [3][z][y][x]); the library copies them
 *     and keeps no reference;
 *   - device memory of a context is either allocated by the library or
 *     supplied by the caller as one workspace (lbs_workspace_bytes); a
 *     supplied workspace stays owned by the caller and must outlive the
 *     context;
 *   - a context is used by one host thread at a time; work is queued on the
 *     context's CUDA stream (borrowed when given, never destroyed);
 *   - lattice units: delta_x = delta_t = 1.
 */
#ifndef LBS_H
#define LBS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LBS_OK = 0,
    LBS_EINVAL = -1,    /* invalid argument or parameter set */
    LBS_ENOMEM = -2,    /* device allocation failed or workspace too small */
    LBS_ECUDA = -3,     /* a CUDA runtime call failed */
    LBS_ENOCONV = -4,   /* SOR did not reach sor_tol within sor_max_iter sweeps */
    LBS_EDIVERGED = -5, /* NaN/Inf in the conserved totals */
    LBS_ETIMEOUT = -6,  /* a bounded device-side wait gave up */
    LBS_EBOUNDS = -7    /* an index check of a debug build failed */
} lbs_status;

/* arithmetic / storage form of the populations and fields */
typedef enum {
    LBS_F64 = 0,  /* everything in double (reference-grade, slow on GB300) */
    LBS_F32 = 1,  /* FP32 storage and arithmetic, FP64 conservation sums */
    LBS_F16 = 2,  /* moving populations stored as IEEE FP16 in shifted form
                     (total minus a rest state, and the minority colour),
                     rounded without bias (to a neighbouring value with
                     probability by distance, drawn from a hash of cell,
                     step and population: reproducible); rest populations in
                     FP32 close each cell's total and minority mass; FP32
                     arithmetic and fields, FP64 totals */
    LBS_BF16 = 3  /* the same with bfloat16 population storage */
} lbs_storage;

/* Physical and numerical parameters (one instance).  Names follow the paper:
 * red = droplet/bubble (rho^N = +1), blue = surfactant-laden liquid. */
typedef struct {
    int nx, ny, nz;           /* grid; nz == 1 selects D2Q9 (2D), nz > 1 D3Q19;
                                 3D: every periodic axis of even length (the
                                 red-black SOR updates in place) */
    int wall[3];              /* per axis: 0 periodic, 1 half-way bounce-back
                                 walls at both ends (Secs. 3.2-3.4, ref. [57]),
                                 2 mirror (symmetry) planes half-way beyond
                                 both ends (Sec. 3.1): specular reflection,
                                 free slip, scalars mirrored, no flux */
    double uw_lo[3][3];       /* velocity of the low wall of each axis (Sec. 3.3) */
    double uw_hi[3][3];       /* velocity of the high wall of each axis */
    double rhoR0, rhoB0;      /* pure-phase densities (Eq. 6) */
    double muR0, muB0;        /* pure-phase dynamic viscosities (Eq. 43) */
    double alphaR, alphaB;    /* sound-speed parameters (App. A, Eq. 42) */
    double sigma0;            /* clean interfacial tension (Eq. 8) */
    double sigma_min_ratio;   /* sigma_min / sigma0, 0.1 in the paper */
    double E0;                /* elasticity number (Eq. 8) */
    double psi_inf;           /* interface capacity psi_infinity (Eq. 8) */
    double beta;              /* recolouring parameter, 0.7 (Eq. 11) */
    int eos;                  /* 0: modified Langmuir (Eq. 8); 1: linear (Sec. 3.2) */
    int source;               /* 0: j of Eq. 22; 1: j = r_a psi_inf C (Sec. 3.1) */
    int transport;            /* 1: solve Eqs. 20-21; 0: hold psi and C fixed */
    double Ds, Db;            /* interface / bulk surfactant diffusivities */
    double ra, rd;            /* adsorption / desorption coefficients (Eq. 22) */
    double g[3];              /* gravity: F_b = (rho - rhoB0) g (Sec. 3.4) */
    double sor_omega;         /* SOR relaxation factor, 1.2 (Sec. 2.2) */
    double sor_tol;           /* stop when max|update| <= sor_tol * max|x| */
    int sor_max_iter;         /* SOR sweeps per solve at most */
    double eps_w;             /* regularisation of the Crank-Nicolson weights */
    double eps_n;             /* regularisation of the interface normal */
} lbs_params;

/* Diagnostics of the current state (Eqs. 33-34 and Sec. 3.4). */
typedef struct {
    double mass_R, mass_B;      /* sum rho^R, sum rho^B (FP64) */
    double surf_total;          /* sum (|grad rhoN|+eps) psi + (1-rhoN+eps) C */
    double surf_pre_rescale;    /* the same total before the last rescale */
    double rescale_factor;      /* factor applied by the last rescale */
    double U[3];                /* mean velocity over rhoN >= 0 (Eqs. 33-34) */
    double centroid[3];         /* centroid of rhoN >= 0 */
    double aspect_ratio;        /* sqrt(I_hh / I_vv), second moments of rhoN >= 0 */
    double psi_av, psi_min, psi_max; /* over cells with |rhoN| < 0.5 */
    double umax;                /* max |u| */
    double Re;                  /* 2 rhoB0 |U_v| R / muB0, R from the red area/volume */
    int sor_iters_psi, sor_iters_C; /* sweeps used by the last solve */
    int sor_rounds;             /* SOR rounds of the last solve: 2D one blocked
                                   launch of 2 sweeps, 3D one red-black sweep */
    long long step;             /* time steps taken since lbs_init_fields */
    double deformation;         /* Taylor deformation (L-B)/(L+B) of rhoN >= 0 from
                                   its principal second moments in the x-y plane
                                   (2D) or x-z plane (3D; Sec. 3.3 shear set-up) */
    double inclination;         /* angle of the major axis from x in that plane (rad) */
} lbs_diag;

typedef struct lbs_ctx lbs_ctx;

/* Fill p with the defaults of the paper (rho 1/1, mu 0.1/0.1, standard
 * alpha, sigma0 0.1, sigma_min 0.1 sigma0, E0 0.5, psi_inf 1, beta 0.7,
 * omega 1.2, D 0.1, periodic walls) for an nx x ny x nz grid. */
int lbs_params_default(lbs_params *p, int nx, int ny, int nz);

/* Device bytes a context needs for p and storage (0 on invalid input). */
size_t lbs_workspace_bytes(const lbs_params *p, int storage);

/* Create a context.  stream: a cudaStream_t to queue work on (borrowed) or
 * NULL for a library-owned stream.  workspace: device memory of at least
 * lbs_workspace_bytes() bytes (caller-owned, 256-byte aligned) or NULL to let
 * the library allocate.  The current CUDA device is used.  Errors:
 * LBS_EINVAL (bad parameters: grid < 3 on a walled axis, non-positive
 * densities or viscosities, ...), LBS_ENOMEM, LBS_ECUDA. */
int lbs_create(const lbs_params *p, int storage, void *stream, void *workspace,
               size_t workspace_bytes, lbs_ctx **out);

/* Initial state from host fields (reading of the paper's initial
 * conditions): colour field phi in [-1, 1] gives rho^R = rhoR0 (1+phi)/2 and
 * rho^B = rhoB0 (1-phi)/2 (so that Eq. 6 returns phi), populations at the
 * equilibrium of App. A with velocity u (NULL = 0); psi, C as given (NULL =
 * 0).  Resets the step counter and the conserved surfactant total. */
int lbs_init_fields(lbs_ctx *c, const double *phi, const double *psi,
                    const double *C, const double *u);

/* Queue n coupled time steps on the context's stream (asynchronous; device
 * errors are reported by the next lbs_sync / lbs_get_fields /
 * lbs_diagnostics).  n >= 0. */
int lbs_step(lbs_ctx *c, int n);

/* Wait for queued work; return the first device-side error (LBS_ENOCONV,
 * LBS_EDIVERGED, LBS_ETIMEOUT) raised since the last check, else LBS_OK. */
int lbs_sync(lbs_ctx *c);

/* Copy the current macroscopic fields to caller-owned host arrays (any may
 * be NULL): density rho = rho^R + rho^B, velocity u of Eq. 10 (3*N),
 * colour field phi = rho^N of Eq. 6, psi, C.  Synchronises. */
int lbs_get_fields(lbs_ctx *c, double *rho, double *u, double *phi,
                   double *psi, double *C);

/* Intermediate fields of the current state, for stage-by-stage checks
 * (any may be NULL; vector fields 3*N): the colour gradient g = grad rho^N
 * (isotropic stencil, Sec. 2.1), a = |grad rho^N|, the total force F of
 * Eq. 9 plus buoyancy, the velocity u of Eq. 10, and the explicit terms
 * S = -div(psi a u) + a j, B = -div(C (1 - rho^N) u) - a j of Eqs. 23-24.
 * Leaves the state unchanged.  Synchronises. */
int lbs_get_macro(lbs_ctx *c, double *g, double *a, double *F, double *u,
                  double *S, double *B);

/* Fill *d with the diagnostics of the current state.  Synchronises. */
int lbs_diagnostics(lbs_ctx *c, lbs_diag *d);

/* ---- measurement ----------------------------------------------------- */

/* Kernel groups of one time step, in launch order.  A 2D context runs the
 * fused step: one launch for force, surfactant terms, collision,
 * recolouring and streaming (timed as LBS_K_COLLIDE) and one for the
 * gradient at t+1, every SOR round, the total and the rescale (timed as
 * LBS_K_SOR; with lbs_set_sor_persistent off, LBS_K_GRAD, LBS_K_SOR and
 * LBS_K_SURF run as launches of their own).  A 3D context runs every group. */
typedef enum {
    LBS_K_FORCE = 0,   /* force and velocity, Eqs. 5-10 */
    LBS_K_FD = 1,      /* explicit surfactant terms and CN right-hand sides */
    LBS_K_COLLIDE = 2, /* collision and recolouring, Eqs. 1-4, 11-12 */
    LBS_K_STREAM = 3,  /* streaming and bounce-back, Eq. 13 */
    LBS_K_GRAD = 4,    /* colour gradient and CN weights at t+1 */
    LBS_K_SOR = 5,     /* all red-black SOR sweeps of the step */
    LBS_K_SURF = 6,    /* total surfactant, rescale, bookkeeping */
    LBS_K_NGROUPS = 7
} lbs_kernel_group;

/* Enable (1) or disable (0) CUDA-event timing of the kernel groups inside
 * the captured step graph (event-record nodes on the context's stream). */
int lbs_profile(lbs_ctx *c, int enable);

/* Synchronise and write, for the most recent step, the device time in
 * milliseconds of each kernel group (ms[LBS_K_NGROUPS]); requires
 * lbs_profile(c, 1) before the steps.  Groups that did not run read 0. */
int lbs_kernel_times(lbs_ctx *c, double *ms, int n);

/* Queue each step as one CUDA graph (enable = 1, the default; the SOR
 * iteration is one cooperative launch, see lbs_set_sor_persistent, or a
 * conditional WHILE node that stops on convergence) or as individual kernel
 * launches with a host-side bound on the SOR rounds (enable = 0, for kernel
 * profilers that cannot trace conditional graphs).  Both forms compute the
 * same numbers. */
int lbs_set_graph(lbs_ctx *c, int enable);

/* Number of kernel launches one step queues (graph kernel nodes). */
int lbs_step_kernel_count(const lbs_ctx *c);

/* ---- total surfactant without any device allocation --------------------
 * (Not part of the paper's method: a service for callers that cannot call
 * cudaMalloc, e.g. code whose device memory belongs to another allocator or
 * a loop that must not stall on an allocation's device synchronisation.)
 *
 * Writes sum (a + eps_w) psi + (chi + eps_w) C over an nx x ny x nz grid to
 * *total, the same conserved total that lbs_diagnostics reports as
 * surf_total when a = |grad rho^N|, chi = 1 - rho^N.  a, chi, psi, C are
 * caller-owned device arrays of float (storage = LBS_F32) or double
 * (LBS_F64), row-major [z][y][x] with a row pitch of `pitch` elements
 * (pitch >= nx); total points to one double the GPU can write (device
 * memory, or mapped / managed host memory).  The work is queued on `stream`
 * (NULL = the legacy default stream); read *total after the stream is
 * synchronised.
 *
 * Nothing is allocated: the per-block partial sums live in a fixed scratch
 * array in the library's device memory (64 KiB, held by every GPU that
 * loads the library until the process exits).  Grids larger than that
 * scratch can serve (more than 8192 thread blocks of 32 x 128 cells; at most
 * LBS_STATIC_MAX_CELLS cells) are refused with LBS_EINVAL before anything is
 * queued.  The first call on a device looks up the scratch's device address;
 * make that first call before any stream capture.  All calls share the
 * scratch: calls that may overlap on the GPU (other streams, other host
 * threads) race and must be serialised by the caller.
 * Returns LBS_OK, LBS_EINVAL (bad arguments, grid too large) or LBS_ECUDA. */
#define LBS_STATIC_MAX_CELLS 33554432LL
int lbs_surfactant_total_static(int storage, const void *a, const void *chi,
                                const void *psi, const void *C, int nx, int ny,
                                int nz, int pitch, double eps_w, double *total,
                                void *stream);

/* Release the context (and its device memory unless caller-supplied). */
void lbs_destroy(lbs_ctx *c);

/* Result of the queued steps for a monitoring loop: waits for the stream
 * (status as lbs_sync), then out[0] = steps taken, out[1] = total surfactant
 * before the last rescale (Sec. 2.2), out[2] = the rescale factor.  A copy
 * of 24 bytes from the context's control block; no kernel is launched. */
int lbs_step_result(lbs_ctx *c, double *out);

/* Blocked SOR tile of a 2D context (Sec. 2.2 solves), as tile / red-black
 * sweeps a launch / threads: 0 = 32x16 / 2 / 256 (default), 1 = 64x8 / 2 /
 * 256, 2 = 16x16 / 2 / 256, 3 = 32x16 / 4 / 256, 4 = 32x32 / 4 / 256,
 * 5 = 32x32 / 4 / 512, 6 = 64x16 / 4 / 512, 7 = 32x32 / 6 / 512,
 * 8 = 32x16 / 8 / 512 (7 and 8 exceed a block's shared memory in FP64 and
 * are refused there).  More sweeps a launch mean fewer launches and a wider
 * halo (2 per sweep); the iterates, and so the results, do not depend on the
 * choice except through where the convergence test falls (after every
 * launch).  3D contexts: 0 = a red and a black half-sweep a sweep, in place,
 * one thread a cell (default), 1 = one full red-black sweep a launch with
 * 32x8 tiles marching through 16-plane chunks of z in shared memory, 2 and
 * 3 = the half-sweeps of 0 with each thread marching a cell pair through 8
 * or 4 planes of z.  Errors: LBS_EINVAL. */
int lbs_set_sor_tile(lbs_ctx *c, int variant);

/* 2D contexts: run the colour gradient at t+1, every round of a solve's
 * blocked SOR (Sec. 2.2), the total surfactant and the rescale in one
 * cooperative launch with grid barriers between them (on, the default; as
 * many blocks as are resident at once, each taking every gridsize-th tile of
 * a round), or the gradient, one launch a round inside the step graph's
 * loop, the total and the rescale as launches of their own (off).  The
 * rounds are the same either way; the totals are summed in different
 * orders, so FP32 results agree to rounding.  In 3D the setting has no
 * effect.  A barrier that waits too long (about a second) reports
 * LBS_ETIMEOUT.  Errors: LBS_EINVAL (no context), LBS_ECUDA. */
int lbs_set_sor_persistent(lbs_ctx *c, int on);

/* The most polls (about 64 ns each) a block of the one-launch SOR waits at
 * the grid barrier between rounds before it gives up: the step then reports
 * LBS_ETIMEOUT (at the next lbs_sync or lbs_diagnostics) instead of waiting
 * on.  Default 2^24, about a second; 0 gives up at once unless every block
 * has arrived.  After a timeout the fields of that step are not valid
 * (initialise them again or load a saved state); the next step's launch
 * starts with a clear barrier.  Errors: LBS_EINVAL (no context, negative limit), LBS_ECUDA. */
int lbs_set_sor_wait_limit(lbs_ctx *c, long long polls);

/* Checkpoint and restart of a single context (Sec. 2.2's time stepping
 * carries state from step to step: the populations of Eq. 13, psi and C,
 * the Adams-Bashforth history S^{t-1}, B^{t-1} of Eqs. 23-24, the conserved
 * total of the rescale and the step counter).  lbs_save_state waits for the
 * queued steps (status as lbs_sync) and writes a raw copy of that state into
 * the caller-owned host buffer buf: a header (grid, storage form, step
 * counter, conserved total M0, last rescale) followed by every carried plane
 * in its stored type (populations in the storage type; fields in the
 * arithmetic type; flags as bytes), dense [z][y][x].  With buf == NULL it
 * only sets *bytes to the size needed; a *bytes below that size gives
 * LBS_EINVAL with *bytes set to the size needed.  On success *bytes is the
 * size written.
 * lbs_load_state copies such a buffer into a context of the same grid and
 * storage form (other parameters may differ) and waits for the copy; the
 * steps that follow give, bit for bit, what the saving context's steps would
 * have given with the same parameters and SOR variant.  Status, arrival
 * counters and SOR progress restart clear.  The buffer is not referenced
 * after the call.
 * Errors: LBS_EINVAL (no context, NULL arguments, buffer too small, a
 * header of another grid, storage form or library version), LBS_ECUDA, or a
 * pending step status (lbs_save_state). */
int lbs_save_state(lbs_ctx *c, void *buf, size_t *bytes);
int lbs_load_state(lbs_ctx *c, const void *buf, size_t bytes);

/* Human-readable description of the last error of c (never NULL). */
const char *lbs_last_error(const lbs_ctx *c);

/* ------------------------------------------------------------------------
 * Batched sweep: n independent 2D instances (each its own lbs_params: grid,
 * Eotvos / Biot numbers, confinement; transport on) advanced together.
 * Each phase of the coupled step is one launch for the whole batch: a grid of
 * (SM count x resident blocks) blocks walks a work list of (instance, tile)
 * items.  The SOR rounds of all instances run in one CUDA-graph WHILE loop,
 * each instance with its own round counter and convergence test (Sec. 2.2
 * tolerance); a converged instance skips the remaining rounds.  One graph
 * holds 8 steps.  Results agree with n single-instance contexts to the
 * rounding of the storage type (the same per-cell bodies, compiled apart). */
typedef struct lbs_batch lbs_batch;

/* Device bytes of the instances' state for p[0..n-1] (0 on invalid input:
 * an invalid instance, nz != 1 or transport == 0). */
size_t lbs_batch_workspace_bytes(const lbs_params *p, int n, int storage);

/* Create a batch of n instances (p: n parameter sets, copied).  stream and
 * workspace as in lbs_create (workspace: lbs_batch_workspace_bytes bytes,
 * caller-owned, 256-byte aligned, or NULL); the work lists and descriptors
 * are allocated by the library.  On failure *out still receives a handle
 * that carries the message (release with lbs_batch_destroy).  Errors:
 * LBS_EINVAL, LBS_ENOMEM, LBS_ECUDA. */
int lbs_batch_create(const lbs_params *p, int n, int storage, void *stream, void *workspace,
                     size_t workspace_bytes, lbs_batch **out);

/* Initial state of instance k (0 <= k < n) from host fields, as
 * lbs_init_fields (arrays of that instance's nx*ny). */
int lbs_batch_init_fields(lbs_batch *b, int k, const double *phi, const double *psi,
                          const double *C, const double *u);

/* Tile shapes: the cell phases run tx x ty thread blocks, one cell per
 * thread (tx*ty a multiple of 32, at most 1024); sor_tile selects the
 * blocked SOR tile and its sweeps a round as lbs_set_sor_tile (0..4).
 * Default 32 x 8, 0.  The cell tile does not change results; the SOR tile
 * only through where the convergence test falls. */
int lbs_batch_set_tiles(lbs_batch *b, int tx, int ty, int sor_tile);

/* Queue n steps of every instance. */
int lbs_batch_step(lbs_batch *b, int n);

/* Wait for queued work; fails with the status of the first instance in the
 * work lists whose solve failed (named in the message). */
int lbs_batch_sync(lbs_batch *b);

/* Fields of instance k, as lbs_get_fields. */
int lbs_batch_get_fields(lbs_batch *b, int k, double *rho, double *u, double *phi, double *psi,
                         double *C);

/* Diagnostics of every instance into d[0..n-1], as lbs_diagnostics. */
int lbs_batch_diagnostics(lbs_batch *b, lbs_diag *d);

/* 1 (default): graphs of 8 steps with the SOR WHILE node; 0: individual
 * launches with a host-driven SOR loop (for kernel profilers). */
int lbs_batch_set_graph(lbs_batch *b, int enable);

/* Kernel launches of one batch step (SOR rounds as of the last diagnostics). */
int lbs_batch_step_kernel_count(const lbs_batch *b);

/* Status of every instance since the last call, status[0..n-1] (lbs_status
 * codes: LBS_EDIVERGED, LBS_ENOCONV, ...), then cleared.  An instance whose
 * total surfactant went non-finite is skipped by every later step (its
 * state is frozen); the others go on.  lbs_batch_sync and
 * lbs_batch_get_fields do not clear these codes; lbs_batch_diagnostics
 * reports every instance and does not fail on them. */
int lbs_batch_status(lbs_batch *b, int *status);

/* Take instance k out of the work lists (active = 0) or back in (1). */
int lbs_batch_set_active(lbs_batch *b, int k, int active);

/* Release the batch (waits for its stream). */
void lbs_batch_destroy(lbs_batch *b);

/* Message of the last failure of a batch. */
const char *lbs_batch_last_error(const lbs_batch *b);

/* ------------------------------------------------------------------------
 * Surrogate network: an ensemble of `members` fully connected networks
 * n_in -> width (depth hidden layers, SiLU) -> n_out (linear), trained by
 * mean-squared error with Adam on the GPU, evaluated with FP32 or bfloat16
 * weights (FP32 arithmetic).  Parameters of a member, FP32: for each layer
 * W (d_out x d_in, row-major) then b (d_out); members follow each other
 * (lbs_mlp_param_count values each).  Host arrays below are caller-owned
 * FP32, row-major, copied in and out; widths are at most 128, depth at
 * most 7.  Errors: LBS_EINVAL (shapes, batch > max_batch, no data set),
 * LBS_ENOMEM, LBS_ECUDA.
 * ---------------------------------------------------------------------- */
typedef struct lbs_mlp lbs_mlp;

/* Create an ensemble (parameters zero until lbs_mlp_init / set_params);
 * max_batch bounds the rows of every call.  stream as in lbs_create. */
int lbs_mlp_create(int members, int n_in, int width, int depth, int n_out, int max_batch,
                   void *stream, lbs_mlp **out);

/* Parameters per member. */
int lbs_mlp_param_count(const lbs_mlp *m);

/* Glorot-uniform weights, zero biases (SplitMix64 on seed and index); resets Adam. */
int lbs_mlp_init(lbs_mlp *m, unsigned long long seed);

/* Copy all members' parameters in / out (members x param_count floats). */
int lbs_mlp_set_params(lbs_mlp *m, const float *params);
int lbs_mlp_get_params(lbs_mlp *m, float *params);

/* Outputs y [members][batch][n_out] of inputs x [members][batch][n_in]
 * (each member its own rows); bf16 != 0: bfloat16 copies of the weights. */
int lbs_mlp_forward(lbs_mlp *m, const float *x, int batch, int bf16, float *y);

/* Loss (mean over rows and outputs of the squared error, per member, FP64
 * out) and its gradient with respect to every parameter (members x
 * param_count, FP32 out; either output may be NULL) for inputs x and
 * targets t [members][batch][n_out].  The gradient is kept for
 * lbs_mlp_adam_step. */
int lbs_mlp_gradient(lbs_mlp *m, const float *x, const float *t, int batch, float *grad,
                     double *loss);

/* Replace the kept gradient (members x param_count floats). */
int lbs_mlp_set_grad(lbs_mlp *m, const float *grad);

/* One Adam step with the kept gradient (Kingma & Ba 2015; bias-corrected). */
int lbs_mlp_adam_step(lbs_mlp *m, float lr, float beta1, float beta2, float eps);

/* Training set X [n][n_in], Y [n][n_out] (copied to the device). */
int lbs_mlp_set_data(lbs_mlp *m, const float *X, const float *Y, int n);

/* iters Adam steps on minibatches of `batch` rows drawn with replacement
 * (SplitMix64 on seed, step, member, row: each member its own rows);
 * loss: the last minibatch's loss per member (may be NULL). */
int lbs_mlp_train(lbs_mlp *m, int iters, int batch, float lr, float beta1, float beta2,
                  float eps, unsigned long long seed, double *loss);

/* Ensemble mean and standard deviation over the members, mean/sd [n][n_out],
 * of the outputs for x [n][n_in] (the same rows for every member). */
int lbs_mlp_predict(lbs_mlp *m, const float *x, int n, int bf16, float *mean, float *sd);

/* Release the ensemble. */
void lbs_mlp_destroy(lbs_mlp *m);

/* Message of the last failure. */
const char *lbs_mlp_last_error(const lbs_mlp *m);

#ifdef __cplusplus
}
#endif
#endif /* LBS_H */
