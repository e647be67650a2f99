/*
 * ora.h — interface of the FP64 CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  The oracle is a plain, slow, step-by-step
 * restatement of the hybrid lattice Boltzmann / finite-difference method for
 * two-phase flow with soluble surfactants (Ba, Liu, Li & Yang, arXiv
 * 2311.15242).  Only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline leg may load it.  It shares no code, header, table or constant
 * generator with the CUDA library (include/lbs.h, paper_2311_15242_gb300/).
 *
 * Conventions
 *   - every floating-point quantity is double;
 *   - fields are row-major [z][y][x] (x fastest), N = nx*ny*nz cells;
 *   - nz == 1 selects the D2Q9 lattice (2D), nz > 1 the D3Q19 lattice (3D);
 *   - lattice units: delta_x = delta_t = 1 (Sec. 2.2 finite differences are
 *     taken on the LB grid).
 */
#ifndef ORA_H
#define ORA_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int nx, ny, nz;
    /* per axis: 0 = periodic, 1 = half-way bounce-back walls at both ends
       (Sec. 3.2, 3.3, 3.4: "half-way bounce-back", ref. [57]), 2 = mirror
       (symmetry) planes half-way beyond both ends (Sec. 3.1: "symmetric
       boundary conditions"; free slip, specular reflection of populations) */
    int wall[3];
    /* velocity vector of the wall at the low / high end of each axis
       (Sec. 3.3: walls moving with opposite velocities) */
    double uw_lo[3][3], uw_hi[3][3];
    /* pure-phase densities, viscosities and sound-speed parameters
       (Eq. 6, Eq. 42, Eq. 43) */
    double rhoR0, rhoB0, muR0, muB0, alphaR, alphaB;
    /* equation of state (Eq. 8): sigma0, sigma_min = ratio*sigma0,
       elasticity E0, capacity psi_inf; recolouring beta (Eq. 11) */
    double sigma0, sigma_min_ratio, E0, psi_inf, beta;
    int eos;        /* 0: modified Langmuir, Eq. 8;  1: linear, Sec. 3.2 */
    int source;     /* 0: j of Eq. 22;  1: j = r_a psi_inf C, Sec. 3.1 */
    int transport;  /* 1: solve Eqs. 20-21;  0: psi and C held fixed */
    double Ds, Db, ra, rd;   /* diffusivities and rate constants, Eqs. 20-22 */
    double g[3];             /* gravity vector: F_b = (rho - rhoB0) g, Sec. 3.4 */
    double sor_omega;        /* 1.2, Sec. 2.2 */
    double sor_tol;          /* stop when max|update| <= tol * max|x| */
    int sor_max_iter;
    double eps_w;            /* regularisation of the CN weights */
    double eps_n;            /* regularisation of the interface normal */
} ora_params;

typedef struct {
    double mass_R, mass_B;           /* sum rho^R, sum rho^B */
    double surf_total;               /* sum a psi + sum chi C (after rescale) */
    double surf_pre_rescale;         /* same sum before the last rescale */
    double rescale_factor;           /* factor applied in the last step */
    double U[3];                     /* droplet velocity, Eqs. 33-34 */
    double centroid[3];
    double aspect_ratio;             /* sqrt(I_xx / I_vv), v = vertical axis */
    double psi_av, psi_min, psi_max; /* over cells with |rho^N| < 0.5 */
    double umax;
    double Re;                       /* 2 rhoB0 U R / muB0 with R from the red area/volume */
    int sor_iters_psi, sor_iters_C;
    long long step;
} ora_diag;

typedef struct ora_ctx ora_ctx;

/* lifecycle (returns NULL / nonzero on invalid parameters) */
ora_ctx *ora_create(const ora_params *p);
void ora_destroy(ora_ctx *o);
int ora_init_fields(ora_ctx *o, const double *phi, const double *psi,
                    const double *C, const double *u /* [3][N] or NULL */);
int ora_step(ora_ctx *o, int n);
/* rho[N], u[3][N], phi[N], psi[N], C[N]; any may be NULL */
int ora_get_fields(ora_ctx *o, double *rho, double *u, double *phi,
                   double *psi, double *C);
int ora_diagnostics(ora_ctx *o, ora_diag *d);
/* raw colour populations fR[Q][N], fB[Q][N] (copies out / in) */
int ora_get_pops(ora_ctx *o, double *fR, double *fB);
int ora_set_pops(ora_ctx *o, const double *fR, const double *fB);
/* set psi and C (after ora_init_fields; also resets the total M0) */
int ora_set_surfactant(ora_ctx *o, const double *psi, const double *C);
long long ora_step_count(const ora_ctx *o);
/* host threads of the cell loops (OpenMP; 1 without it).  n > 0 sets the
   count for the process; returns the count in use.  Results do not depend
   on it: only loops whose cells are independent are shared out. */
int ora_threads(int n);

/* intermediate fields of one step at the current state, each [N] unless
   noted: rhoR, rhoB, rhoN, g[3][N] (colour gradient), a (=|grad rhoN|),
   kappa, F[3][N] (total force), u[3][N], S, B (explicit FD terms of
   Eqs. 23-24 at the current time level).  Any may be NULL. */
int ora_macro(ora_ctx *o, double *rhoR, double *rhoB, double *rhoN, double *g,
              double *a, double *kappa, double *F, double *u, double *S,
              double *B);

/* ---- building blocks, exported for the pins in tests/ ---- */
int ora_lattice(int D, int *Q, int *e /* [Q][3] */, double *w /* [Q] */,
                double *M /* [Q][Q] */, double *Minv /* [Q][Q] */);
/* moment-space equilibria m^{k,eq} of one colour, Eq. 37 (D=2) / Eq. 40 (D=3) */
void ora_meq(int D, double rho_k, const double *u, double alpha_k, double *m);
/* correction term C^k in moment space from Q = (Q_x, Q_y, Q_z) */
void ora_corr(int D, const double *Qv, double *c);
/* relaxation diagonal S, Eq. 38 / Eq. 41 */
void ora_relax(int D, double s_v, double *S);
/* forcing moments F_j of Eq. 4 */
void ora_forcing(int D, const double *u, const double *F, double *Fh);
/* sound-speed squared of a colour with parameter alpha, App. A */
double ora_cs2(int D, double alpha);
/* one-cell collision (Eqs. 1-4) followed by recolouring (Eqs. 11-12).
   fR, fB: pre-collision colour populations [Q]; u, F: velocity and force;
   dRu, dBu: isotropic derivatives d_alpha(rho^k u_alpha) of each colour
   (3 values each); g: colour gradient.  Outputs post-recolouring fR2, fB2. */
void ora_collide_cell(const ora_params *p, int D, const double *fR,
                      const double *fB, const double *u, const double *F,
                      const double *dRu, const double *dBu, const double *g,
                      double *fR2, double *fB2);
/* equation of state, Eq. 8 (or the linear law): sigma and the Marangoni
   coefficient -d sigma / d psi used in Eq. 9 (0 at or above the CMC) */
void ora_eos(const ora_params *p, double psi, double *sigma, double *mcoef);
double ora_cmc(const ora_params *p);
/* finite-difference operators on a field of the context's grid */
int ora_iso_grad(ora_ctx *o, const double *x, double *grad /* [3][N] */);
/* div Psi with the WENO3 one-sided differences of Eqs. 25-27;
   Psi[3][N], u[3][N] selects the upwind side */
int ora_weno_div(ora_ctx *o, const double *Psi, const double *u, double *div);
/* Eq. 28: L_w x = sum_faces w_face (x_nb - x_c) */
int ora_diffuse(ora_ctx *o, const double *w, const double *x, double *Lx);
/* SOR (Sec. 2.2) for (w - h L_w) x = rhs; x holds the initial guess on
   entry and the solution on exit; returns sweeps used or -1 on no
   convergence */
int ora_sor(ora_ctx *o, const double *w, double h, const double *rhs,
            double *x);

/* ---- a step in phases, for a grid decomposed into slabs along its slowest
   axis (rows: y in 2D, z in 3D); one_step is exactly these in order ---- */
/* boundaries of the two ends of axis a: 0 periodic wrap, 1 bounce-back wall,
   2 mirror plane (default: both ends as wall[a]) */
int ora_set_ends(ora_ctx *o, int a, int lo, int hi);
/* k = 0: fields at t, explicit terms, collision, streaming; 1: the
   Crank-Nicolson right-hand sides (weights of t); 2: fields at t+1; 3, 4:
   the SOR weights of psi, of C */
int ora_phase(ora_ctx *o, int k);
/* one lexicographic SOR sweep of psi (which 0) or C (1) over rows [r0, r1),
   folding the largest update and |x| into *maxd, *maxx */
int ora_sor_rows(ora_ctx *o, int which, int r0, int r1, double *maxd, double *maxx);
/* continue the Kahan-compensated total surfactant ks = {sum, compensation}
   over rows [r0, r1) */
int ora_surf_rows(ora_ctx *o, int r0, int r1, double *ks);
/* rescale psi and C by s, keep S, B as the history, count the step */
int ora_finish(ora_ctx *o, double s, double pre, int itp, int itc);
void ora_set_M0(ora_ctx *o, double M0);
/* the context's own arrays: fR, fB ([Q][N]), psi, C, Sp, Bp, a, rhoN */
double *ora_field(ora_ctx *o, const char *name);

#ifdef __cplusplus
}
#endif
#endif
