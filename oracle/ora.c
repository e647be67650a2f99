/*
 * ora.c — FP64 CPU oracle of the hybrid LB-FD coupled step.
 *
 * TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and bench.py's
 * CPU-baseline leg are the only users.  Plain loops, one field at a time, in
 * the order the paper describes the method (arXiv 2311.15242):
 *
 *   Sec. 2.1  lattice Boltzmann colour-gradient model
 *             Eq. 1-4   MRT collision with correction and forcing terms
 *             Eq. 5-9   interfacial force from the modified Langmuir EOS
 *             Eq. 10    velocity with the half-force shift
 *             Eq. 11-12 recolouring;  Eq. 13 streaming
 *             App. A    Eq. 36-43 lattice matrices, equilibria, relaxation
 *   Sec. 2.2  finite differences for the surfactant equations
 *             Eq. 20-22 diffuse-interface equations and source term
 *             Eq. 23-24 modified Crank-Nicolson / Adams-Bashforth in time
 *             Eq. 25-27 WENO3 convection;  Eq. 28 diffusion operator
 *             SOR (omega = 1.2) and the rescaling of the total surfactant
 *
 * Readings of points the paper leaves open (numbered R1..R28) are marked
 * "reading:" where they are used.
 *
 * Parity unpinned: the velocity terms of the D3Q19 equilibrium rows 17-19
 * (Eq. 40, taken as printed) have no independent check (their rest value
 * is checked against the alpha-model's rest state); the 3D correction
 * coefficient is checked only where it vanishes (standard alpha).
 */
#include "ora.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define QMAX 19
#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif
#define CS2 (1.0 / 3.0) /* lattice sound speed squared of Eq. 4 (Sec. 2.1) */
#define WENO_EPS 1e-6   /* epsilon of the WENO weights, Sec. 2.2 */

/* ------------------------------------------------------------------------
 * Lattices.  Reading: the velocity order is the one implied by the rows of
 * M that carry the momentum (rows 4, 6 of Eq. 36; rows 2-4 of Eq. 39); the
 * weights are the standard D2Q9 / D3Q19 ones (the paper cites [42, 45]).
 * ---------------------------------------------------------------------- */
static const int E2[9][3] = {{0, 0, 0},  {1, 0, 0},  {0, 1, 0},
                             {-1, 0, 0}, {0, -1, 0}, {1, 1, 0},
                             {-1, 1, 0}, {-1, -1, 0}, {1, -1, 0}};
static const double W2[9] = {4.0 / 9,  1.0 / 9,  1.0 / 9,  1.0 / 9, 1.0 / 9,
                             1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
/* Eq. 36 */
static const double M2[9][9] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1},         {-4, -1, -1, -1, -1, 2, 2, 2, 2},
    {4, -2, -2, -2, -2, 1, 1, 1, 1},     {0, 1, 0, -1, 0, 1, -1, -1, 1},
    {0, -2, 0, 2, 0, 1, -1, -1, 1},      {0, 0, 1, 0, -1, 1, 1, -1, -1},
    {0, 0, -2, 0, 2, 1, 1, -1, -1},      {0, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 1, -1, 1, -1}};

static const int E3[19][3] = {
    {0, 0, 0},   {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},   {0, -1, 0},
    {0, 0, 1},   {0, 0, -1},  {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
    {-1, 1, 0},  {1, 0, 1},   {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1},   {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
static const double W3[19] = {1.0 / 3,  1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18,
                              1.0 / 18, 1.0 / 18, 1.0 / 36, 1.0 / 36, 1.0 / 36,
                              1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36,
                              1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
/* Eq. 39 */
static const double M3[19][19] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1},
    {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1},
    {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1},
    {0, 1, 1, 1, 1, 1, 1, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2},
    {0, 2, 2, -1, -1, -1, -1, 1, 1, 1, 1, 1, 1, 1, 1, -2, -2, -2, -2},
    {0, 0, 0, 1, 1, -1, -1, 1, 1, 1, 1, -1, -1, -1, -1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, -1, -1},
    {0, 0, 0, 0, 0, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 0, 0, 1, -1, 1, -1, 0, 0, 0, 0, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, -1, -1, 1},
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, -1, 1, -1},
    {0, 0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 0, 0, 0, 0, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, 1, 1}};

/* Gauss-Jordan inverse with partial pivoting (M^{-1} of Eq. 2, 3) */
static int invert(int n, const double *A, double *Ainv) {
    double a[QMAX][2 * QMAX];
    for (int i = 0; i < n; i++)
        for (int j = 0; j < 2 * n; j++)
            a[i][j] = j < n ? A[i * n + j] : (j - n == i ? 1.0 : 0.0);
    for (int c = 0; c < n; c++) {
        int piv = c;
        for (int r = c + 1; r < n; r++)
            if (fabs(a[r][c]) > fabs(a[piv][c])) piv = r;
        if (fabs(a[piv][c]) < 1e-14) return -1;
        if (piv != c)
            for (int j = 0; j < 2 * n; j++) {
                double t = a[c][j];
                a[c][j] = a[piv][j];
                a[piv][j] = t;
            }
        double d = a[c][c];
        for (int j = 0; j < 2 * n; j++) a[c][j] /= d;
        for (int r = 0; r < n; r++) {
            if (r == c || a[r][c] == 0.0) continue;
            double f = a[r][c];
            for (int j = 0; j < 2 * n; j++) a[r][j] -= f * a[c][j];
        }
    }
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) Ainv[i * n + j] = a[i][n + j];
    return 0;
}

/* lattice tables of one dimension, filled on first use */
typedef struct {
    int q;
    int e[QMAX * 3];
    double w[QMAX], M[QMAX * QMAX], Minv[QMAX * QMAX];
    int ok;
} lattice_t;

static const lattice_t *lat(int D) {
    static lattice_t L[2];
    lattice_t *l = &L[D == 2 ? 0 : 1];
    if (l->ok) return l;
    l->q = D == 2 ? 9 : 19;
    for (int i = 0; i < l->q; i++) {
        for (int a = 0; a < 3; a++) l->e[i * 3 + a] = D == 2 ? E2[i][a] : E3[i][a];
        l->w[i] = D == 2 ? W2[i] : W3[i];
        for (int j = 0; j < l->q; j++)
            l->M[i * l->q + j] = D == 2 ? M2[i][j] : M3[i][j];
    }
    if (invert(l->q, l->M, l->Minv) == 0) l->ok = 1;
    return l;
}

int ora_lattice(int D, int *Q, int *e, double *w, double *M, double *Minv) {
    if (D != 2 && D != 3) return -1;
    const lattice_t *l = lat(D);
    if (!l->ok) return -1;
    int q = l->q;
    if (Q) *Q = q;
    if (e) memcpy(e, l->e, sizeof(int) * 3 * q);
    if (w) memcpy(w, l->w, sizeof(double) * q);
    if (M) memcpy(M, l->M, sizeof(double) * q * q);
    if (Minv) memcpy(Minv, l->Minv, sizeof(double) * q * q);
    return 0;
}

/* (c_s^k)^2 = (3/5)(1 - alpha^k) in 2D, (1/2)(1 - alpha^k) in 3D (App. A) */
double ora_cs2(int D, double alpha) {
    return D == 2 ? 0.6 * (1.0 - alpha) : 0.5 * (1.0 - alpha);
}

/* moment-space equilibrium of one colour: Eq. 37 (2D), Eq. 40 (3D) */
void ora_meq(int D, double r, const double *u, double al, double *m) {
    double ux = u[0], uy = u[1], uz = D == 3 ? u[2] : 0.0;
    if (D == 2) {
        double u2 = ux * ux + uy * uy;
        m[0] = r;
        m[1] = r * (-3.6 * al - 0.4 + 3.0 * u2);
        m[2] = r * (5.4 * al - 1.4 - 3.0 * u2);
        m[3] = r * ux;
        m[4] = r * (-1.8 * al - 0.2) * ux;
        m[5] = r * uy;
        m[6] = r * (-1.8 * al - 0.2) * uy;
        m[7] = r * (ux * ux - uy * uy);
        m[8] = r * ux * uy;
        return;
    }
    double u2 = ux * ux + uy * uy + uz * uz;
    double p = r * ora_cs2(3, al); /* p^k = rho^k (c_s^k)^2 */
    m[0] = r;
    m[1] = r * ux;
    m[2] = r * uy;
    m[3] = r * uz;
    m[4] = 3.0 * p + r * u2;
    m[5] = r * (2.0 * ux * ux - uy * uy - uz * uz);
    m[6] = r * (uy * uy - uz * uz);
    m[7] = r * ux * uy;
    m[8] = r * ux * uz;
    m[9] = r * uy * uz;
    m[10] = p * uy;
    m[11] = p * ux;
    m[12] = p * uz;
    m[13] = p * ux;
    m[14] = p * uz;
    m[15] = p * uy;
    /* rows 17-19 as printed in Eq. 40 (reading R7) */
    m[16] = r * ((1.0 - al - u2) + 2.0 * (ux * ux + uy * uy)) / 6.0;
    m[17] = r * ((1.0 - al - u2) + 2.0 * (ux * ux + uz * uz)) / 6.0;
    m[18] = r * ((1.0 - al - u2) + 2.0 * (uy * uy + uz * uz)) / 6.0;
}

/* correction term C^k: Eq. 37 (2D) / Eq. 40 (3D) */
void ora_corr(int D, const double *Qv, double *c) {
    int q = D == 2 ? 9 : 19;
    for (int j = 0; j < q; j++) c[j] = 0.0;
    if (D == 2) {
        c[1] = 3.0 * Qv[0] + 3.0 * Qv[1];
        c[7] = Qv[0] - Qv[1];
        return;
    }
    c[4] = Qv[0] + Qv[1] + Qv[2];
    c[5] = 2.0 * Qv[0] - Qv[1] - Qv[2];
    c[6] = Qv[1] - Qv[2];
}

/* relaxation matrix diagonal: Eq. 38 (2D), Eq. 41 (3D) */
void ora_relax(int D, double sv, double *S) {
    if (D == 2) {
        const double s[9] = {0, 1.25, 1.14, 0, 1.6, 0, 1.6, 0, 0};
        for (int j = 0; j < 9; j++) S[j] = s[j];
        S[7] = sv;
        S[8] = sv;
        return;
    }
    for (int j = 0; j < 19; j++) S[j] = 1.0;
    for (int j = 5; j <= 9; j++) S[j] = sv;
}

/* forcing moments F_j = sum_k M_jk w_k [(e_k-u)/cs2 + (e_k.u) e_k/cs2^2].F (Eq. 4) */
void ora_forcing(int D, const double *u, const double *F, double *Fh) {
    const lattice_t *l = lat(D);
    const int q = l->q, *e = l->e;
    const double *w = l->w, *M = l->M;
    double gk[QMAX];
    for (int k = 0; k < q; k++) {
        double eu = 0, eF = 0, uF = 0;
        for (int a = 0; a < D; a++) {
            eu += e[k * 3 + a] * u[a];
            eF += e[k * 3 + a] * F[a];
            uF += u[a] * F[a];
        }
        gk[k] = w[k] * ((eF - uF) / CS2 + eu * eF / (CS2 * CS2));
    }
    for (int j = 0; j < q; j++) {
        double s = 0;
        for (int k = 0; k < q; k++) s += M[j * q + k] * gk[k];
        Fh[j] = s;
    }
}

/* ------------------------------------------------------------------------
 * Equation of state, Eq. 8, and the coefficient -d sigma/d psi of Eq. 9.
 * Reading R15: the CMC test is taken before the logarithm, which is never
 * evaluated at or above the CMC; ln(1 - psi/psi_inf) is log1p(-psi/psi_inf).
 * ---------------------------------------------------------------------- */
double ora_cmc(const ora_params *p) {
    if (p->eos != 0 || p->E0 <= 0.0) return HUGE_VAL;
    /* sigma_min = ratio*sigma0 => CMC = psi_inf [1 - exp(-(1-ratio)/E0)];
       with ratio = 1/10 this is psi_inf [1 - exp(-0.9/E0)] (Sec. 2.1) */
    return p->psi_inf * (1.0 - exp(-(1.0 - p->sigma_min_ratio) / p->E0));
}

void ora_eos(const ora_params *p, double psi, double *sigma, double *mcoef) {
    if (p->eos == 1) { /* linear law of Sec. 3.2 */
        *sigma = p->sigma0 * (1.0 - p->E0 * psi / p->psi_inf);
        *mcoef = p->sigma0 * p->E0 / p->psi_inf;
        return;
    }
    if (p->E0 == 0.0) { /* Eq. 8 with E0 = 0: sigma = sigma0 for every psi */
        *sigma = p->sigma0;
        *mcoef = 0.0;
        return;
    }
    if (psi < ora_cmc(p)) {
        *sigma = p->sigma0 * (1.0 + p->E0 * log1p(-psi / p->psi_inf));
        *mcoef = p->sigma0 * p->E0 / (p->psi_inf - psi);
    } else {
        *sigma = p->sigma_min_ratio * p->sigma0;
        *mcoef = 0.0;
    }
}

/* one-cell collision (Eqs. 1-4 with App. A) and recolouring (Eqs. 11-12) */
void ora_collide_cell(const ora_params *p, int D, const double *fR,
                      const double *fB, const double *u, const double *F,
                      const double *dRu, const double *dBu, const double *g,
                      double *fR2, double *fB2) {
    const lattice_t *l = lat(D);
    const int q = l->q, *e = l->e;
    const double *M = l->M, *Minv = l->Minv;

    double rR = 0, rB = 0;
    for (int i = 0; i < q; i++) {
        rR += fR[i];
        rB += fB[i];
    }
    double rho = rR + rB;
    /* colour function, Eq. 6 */
    double xr = rR / p->rhoR0, xb = rB / p->rhoB0;
    double rN = (xr - xb) / (xr + xb);

    /* m = M f of the total distribution (Eq. 2) */
    double m[QMAX], meqR[QMAX], meqB[QMAX], cR[QMAX], cB[QMAX], Fh[QMAX],
        S[QMAX], ms[QMAX];
    for (int j = 0; j < q; j++) {
        double s = 0;
        for (int i = 0; i < q; i++) s += M[j * q + i] * (fR[i] + fB[i]);
        m[j] = s;
    }
    ora_meq(D, rR, u, p->alphaR, meqR);
    ora_meq(D, rB, u, p->alphaB, meqB);

    /* Q^k: 2D (1.8 alpha^k - 0.8) d_a(rho^k u_a) (App. A); 3D reading R6:
       d_a{rho^k u_a [1 - 3 (c_s^k)^2]} */
    double coefR, coefB, QR[3] = {0, 0, 0}, QB[3] = {0, 0, 0};
    if (D == 2) {
        coefR = 1.8 * p->alphaR - 0.8;
        coefB = 1.8 * p->alphaB - 0.8;
    } else {
        coefR = 1.0 - 3.0 * ora_cs2(3, p->alphaR);
        coefB = 1.0 - 3.0 * ora_cs2(3, p->alphaB);
    }
    for (int a = 0; a < D; a++) {
        QR[a] = coefR * dRu[a];
        QB[a] = coefB * dBu[a];
    }
    ora_corr(D, QR, cR);
    ora_corr(D, QB, cB);
    ora_forcing(D, u, F, Fh);

    /* mixture viscosity, Eq. 43, and s_v from mu = (1/s_v - 1/2) sum_k rho^k (c_s^k)^2 */
    double inv_mu = (1.0 + rN) / (2.0 * p->muR0) + (1.0 - rN) / (2.0 * p->muB0);
    double mu = 1.0 / inv_mu;
    double pk = rR * ora_cs2(D, p->alphaR) + rB * ora_cs2(D, p->alphaB);
    double sv = 1.0 / (0.5 + mu / pk);
    ora_relax(D, sv, S);

    /* f^dagger = f + M^{-1}[-S(m - m^eq) + (I - S/2)(C + F)]  (Eqs. 1-3) */
    for (int j = 0; j < q; j++)
        ms[j] = m[j] - S[j] * (m[j] - meqR[j] - meqB[j]) +
                (1.0 - 0.5 * S[j]) * (cR[j] + cB[j] + Fh[j]);
    double fd[QMAX];
    for (int i = 0; i < q; i++) {
        double s = 0;
        for (int j = 0; j < q; j++) s += Minv[i * q + j] * ms[j];
        fd[i] = s;
    }

    /* recolouring, Eqs. 11-12.  cos(theta_i)|e_i| = e_i.grad rhoN / |grad rhoN|;
       reading R3: |grad rhoN| -> sqrt(|grad rhoN|^2 + eps_n^2).
       Reading R23: the weight w_i of Eq. 11 is the rest-state weight of the
       equilibrium, f_i^eq(rho, u=0)/rho with f^eq(0) = sum_k M^{-1} m^{k,eq}(rho^k, 0);
       it equals w_i on the standard lattice (equal densities) and keeps the
       colour populations non-negative for the alpha-model at unequal densities. */
    double feq0[QMAX], mzR[QMAX], mzB[QMAX];
    const double zero[3] = {0, 0, 0};
    ora_meq(D, rR, zero, p->alphaR, mzR);
    ora_meq(D, rB, zero, p->alphaB, mzB);
    for (int i = 0; i < q; i++) {
        double s = 0;
        for (int j = 0; j < q; j++) s += Minv[i * q + j] * (mzR[j] + mzB[j]);
        feq0[i] = s;
    }
    double gn = 0;
    for (int a = 0; a < D; a++) gn += g[a] * g[a];
    gn = sqrt(gn + p->eps_n * p->eps_n);
    for (int i = 0; i < q; i++) {
        double eg = 0;
        for (int a = 0; a < D; a++) eg += e[i * 3 + a] * g[a];
        double seg = p->beta * (feq0[i] / rho) * rR * rB / rho * eg / gn;
        fR2[i] = rR / rho * fd[i] + seg;
        fB2[i] = rB / rho * fd[i] - seg;
    }
}

/* ------------------------------------------------------------------------
 * Context and grid helpers
 * ---------------------------------------------------------------------- */
struct ora_ctx {
    ora_params p;
    int D, Q;
    long N;
    int e[QMAX][3], opp[QMAX];
    int mir[8][QMAX];              /* direction mirrored on the axes of a bit mask */
    double w[QMAX];
    double *fR, *fB, *fR2, *fB2;   /* [Q][N] */
    double *psi, *C, *Sp, *Bp;     /* [N] */
    /* work fields */
    double *rhoR, *rhoB, *rho, *rhoN, *g, *a, *n, *kap, *F, *u, *gpsi;
    double *S, *B, *rhs, *wt, *tmp, *Psi;
    long *face;                    /* [2D][N] face neighbours, -1 = wall */
    /* boundary of each end of each axis: 0 periodic wrap, 1 bounce-back
       wall, 2 mirror plane; both ends follow p.wall unless a slab of a
       decomposed grid sets them (ora_set_ends) */
    int end[3][2];
    long long step;
    double M0;
    double last_pre, last_scale;
    int last_it_psi, last_it_C;
};

static long idx(const ora_ctx *o, int x, int y, int z) {
    return ((long)z * o->p.ny + y) * o->p.nx + x;
}

/* Neighbour of (x,y,z) at offset d.  Periodic axes wrap.  On walled axes
   the coordinate is mirrored about the half-way wall (-1 -> 0, -2 -> 1,
   n -> n-1, ...); bit a of *refl marks a reflection on axis a and side[a]
   is -1 for the low wall, +1 for the high wall. */
static long nb(const ora_ctx *o, int x, int y, int z, const int *d, int *refl,
               int *side) {
    int c[3] = {x + d[0], y + d[1], z + d[2]};
    int n[3] = {o->p.nx, o->p.ny, o->p.nz};
    *refl = 0;
    if (c[0] >= 0 && c[0] < n[0] && c[1] >= 0 && c[1] < n[1] && c[2] >= 0 &&
        c[2] < n[2]) {
        side[0] = side[1] = side[2] = 0;
        return idx(o, c[0], c[1], c[2]);
    }
    for (int a = 0; a < 3; a++) {
        side[a] = 0;
        if (c[a] >= 0 && c[a] < n[a]) continue;
        if (!o->end[a][c[a] < 0 ? 0 : 1]) {
            c[a] = ((c[a] % n[a]) + n[a]) % n[a];
            continue;
        }
        *refl |= 1 << a;
        if (c[a] < 0) {
            side[a] = -1;
            c[a] = -1 - c[a];
        } else {
            side[a] = 1;
            c[a] = 2 * n[a] - 1 - c[a];
        }
    }
    return idx(o, c[0], c[1], c[2]);
}

/* velocity seen at a ghost node (reading R21): for each wall crossed,
   u -> 2 u_wall - u, i.e. linear in the normal direction with the wall
   velocity half-way (no-slip, half-way bounce-back); for each mirror plane
   crossed, the mirror image: the normal component changes sign, the
   tangential ones are kept (free slip) */
static void ghost_u(const ora_ctx *o, const double *u, long j, int refl,
                    const int *side, double *out) {
    for (int b = 0; b < 3; b++) out[b] = u[b * o->N + j];
    for (int a = 0; a < 3; a++) {
        if (!(refl & (1 << a))) continue;
        if (o->end[a][side[a] < 0 ? 0 : 1] == 2) {
            out[a] = -out[a];
            continue;
        }
        const double *uw = side[a] < 0 ? o->p.uw_lo[a] : o->p.uw_hi[a];
        for (int b = 0; b < 3; b++) out[b] = 2.0 * uw[b] - out[b];
    }
}

#define FOR_CELLS(o)                          \
    for (int z = 0; z < (o)->p.nz; z++)       \
        for (int y = 0; y < (o)->p.ny; y++)   \
            for (int x = 0; x < (o)->p.nx; x++)

/* The same loops shared out over the host's threads (OpenMP, when built
   with it).  Used only where every cell writes its own outputs and reads
   nothing written in the same loop, so the results do not depend on the
   thread count; sums and the lexicographic SOR stay sequential. */
#define PAR_CELLS(o) _Pragma("omp parallel for collapse(2) schedule(static)") FOR_CELLS(o)
#define PAR_FOR _Pragma("omp parallel for schedule(static)")

/* isotropic finite-difference gradient (Sec. 2.1 after Eq. 9, ref. [40]);
   reading R2: d_a X(x) = (1/cs2) sum_i w_i X(x + e_i) e_ia.
   Scalars are mirrored (even) at walls (reading R21). */
static void grad_scalar(const ora_ctx *o, const double *X, double *G) {
    PAR_CELLS(o) {
        long c = idx(o, x, y, z);
        double s[3] = {0, 0, 0};
        for (int i = 1; i < o->Q; i++) {
            int refl, side[3];
            long j = nb(o, x, y, z, o->e[i], &refl, side);
            for (int a = 0; a < 3; a++) s[a] += o->w[i] * X[j] * o->e[i][a];
        }
        for (int a = 0; a < 3; a++) G[a * o->N + c] = s[a] / CS2;
    }
}

int ora_iso_grad(ora_ctx *o, const double *x, double *grad) {
    grad_scalar(o, x, grad);
    return 0;
}

/* ------------------------------------------------------------------------
 * Macroscopic quantities of one time level (Sec. 2.1)
 * ---------------------------------------------------------------------- */
static void macro(ora_ctx *o, const double *fR, const double *fB,
                  const double *psi) {
    const ora_params *p = &o->p;
    long N = o->N;
    int D = o->D;
    /* colour densities and colour function, Eq. 6 (rho^k = sum_i f_i^k) */
    PAR_FOR for (long c = 0; c < N; c++) {
        double r = 0, b = 0;
        for (int i = 0; i < o->Q; i++) {
            r += fR[i * N + c];
            b += fB[i * N + c];
        }
        o->rhoR[c] = r;
        o->rhoB[c] = b;
        o->rho[c] = r + b;
        double xr = r / p->rhoR0, xb = b / p->rhoB0;
        o->rhoN[c] = (xr - xb) / (xr + xb);
    }
    /* colour gradient, its magnitude and the unit normal n = -grad/|grad|
       (after Eq. 6); reading R3 regularises the normalisation */
    grad_scalar(o, o->rhoN, o->g);
    PAR_FOR for (long c = 0; c < N; c++) {
        double s = 0;
        for (int a = 0; a < 3; a++) s += o->g[a * N + c] * o->g[a * N + c];
        o->a[c] = sqrt(s);
        double gn = sqrt(s + p->eps_n * p->eps_n);
        for (int a = 0; a < 3; a++) o->n[a * N + c] = -o->g[a * N + c] / gn;
    }
    /* curvature kappa = -div n, Eq. 7, with the isotropic derivative; at a
       wall the normal component of n is mirrored with a sign change */
    PAR_CELLS(o) {
        long c = idx(o, x, y, z);
        double s = 0;
        for (int i = 1; i < o->Q; i++) {
            int refl, side[3];
            long j = nb(o, x, y, z, o->e[i], &refl, side);
            for (int a = 0; a < D; a++) {
                double v = o->n[a * N + j];
                if (refl & (1 << a)) v = -v;
                s += o->w[i] * v * o->e[i][a];
            }
        }
        o->kap[c] = -s / CS2;
    }
    /* interfacial force, Eq. 9, plus buoyancy F_b = (rho - rhoB0) g (Sec. 3.4) */
    grad_scalar(o, psi, o->gpsi);
    double cmc = ora_cmc(p);
    PAR_FOR for (long c = 0; c < N; c++) {
        double sig, mco;
        ora_eos(p, psi[c], &sig, &mco);
        double F[3];
        if (psi[c] < cmc) {
            double ndg = 0;
            for (int a = 0; a < 3; a++) ndg += o->n[a * N + c] * o->gpsi[a * N + c];
            for (int a = 0; a < 3; a++)
                F[a] = -0.5 * sig * o->kap[c] * o->g[a * N + c] -
                       0.5 * o->a[c] * mco *
                           (o->gpsi[a * N + c] - ndg * o->n[a * N + c]);
        } else {
            for (int a = 0; a < 3; a++)
                F[a] = -0.5 * p->sigma_min_ratio * p->sigma0 * o->kap[c] *
                       o->g[a * N + c];
        }
        for (int a = 0; a < 3; a++) {
            F[a] += (o->rho[c] - p->rhoB0) * p->g[a];
            if (a >= D) F[a] = 0.0;
            o->F[a * N + c] = F[a];
        }
    }
    /* velocity with the half-force shift, Eq. 10 (F = F_s + F_b) */
    PAR_FOR for (long c = 0; c < N; c++) {
        double j[3] = {0, 0, 0};
        for (int i = 0; i < o->Q; i++) {
            double f = fR[i * N + c] + fB[i * N + c];
            for (int a = 0; a < 3; a++) j[a] += f * o->e[i][a];
        }
        for (int a = 0; a < 3; a++)
            o->u[a * N + c] = (j[a] + 0.5 * o->F[a * N + c]) / o->rho[c];
    }
}

/* ------------------------------------------------------------------------
 * Finite differences of Sec. 2.2
 * ---------------------------------------------------------------------- */

/* WENO3 one-sided differences, Eqs. 26-27, on the values v[-2..2] around
   node i (v points at v_i).  D^- uses {i-2..i+1}, D^+ uses {i-1..i+2}. */
static double dplus(const double *v, int k) { return v[k + 1] - v[k]; }
static double d2(const double *v, int k) { return v[k + 1] - 2.0 * v[k] + v[k - 1]; }

static double weno_minus(const double *v) {
    double r = (WENO_EPS + d2(v, -1) * d2(v, -1)) / (WENO_EPS + d2(v, 0) * d2(v, 0));
    double wm = 1.0 / (1.0 + 2.0 * r * r);
    return 0.5 * ((dplus(v, -1) + dplus(v, 0)) -
                  wm * (dplus(v, -2) - 2.0 * dplus(v, -1) + dplus(v, 0)));
}

static double weno_plus(const double *v) {
    double r = (WENO_EPS + d2(v, 1) * d2(v, 1)) / (WENO_EPS + d2(v, 0) * d2(v, 0));
    double wp = 1.0 / (1.0 + 2.0 * r * r);
    return 0.5 * ((dplus(v, -1) + dplus(v, 0)) -
                  wp * (dplus(v, 1) - 2.0 * dplus(v, 0) + dplus(v, -1)));
}

/* div Psi by Eq. 25.  Reading R9: along axis d the left-biased D^- is used
   where u_d > 0, the right-biased D^+ where u_d < 0, and their mean where
   u_d = 0.  At a wall Psi_d (normal flux) is mirrored with a sign change. */
static void weno_div(const ora_ctx *o, const double *Psi, const double *u,
                     double *div) {
    long N = o->N;
    PAR_CELLS(o) {
        long c = idx(o, x, y, z);
        double s = 0;
        for (int d = 0; d < o->D; d++) {
            double vv[5];
            for (int k = -2; k <= 2; k++) {
                int off[3] = {0, 0, 0}, refl, side[3];
                off[d] = k;
                long j = nb(o, x, y, z, off, &refl, side);
                double v = Psi[d * N + j];
                if (refl & (1 << d)) v = -v;
                vv[k + 2] = v;
            }
            const double *v = vv + 2;
            double ud = u[d * N + c];
            if (ud > 0)
                s += weno_minus(v);
            else if (ud < 0)
                s += weno_plus(v);
            else
                s += 0.5 * (weno_minus(v) + weno_plus(v));
        }
        div[c] = s;
    }
}

int ora_weno_div(ora_ctx *o, const double *Psi, const double *u, double *div) {
    weno_div(o, Psi, u, div);
    return 0;
}

/* Eq. 28: sum over faces of w_face (X_nb - X_c), w_face = (w_c + w_nb)/2.
   Reading R21: a face on a wall carries no flux. */
static void diffuse(const ora_ctx *o, const double *W, const double *X,
                    double *L) {
    PAR_FOR for (long c = 0; c < o->N; c++) {
        double s = 0;
        for (int f = 0; f < 2 * o->D; f++) {
            long j = o->face[f * o->N + c];
            if (j < 0) continue;
            s += 0.5 * (W[c] + W[j]) * (X[j] - X[c]);
        }
        L[c] = s;
    }
}

int ora_diffuse(ora_ctx *o, const double *w, const double *x, double *Lx) {
    diffuse(o, w, x, Lx);
    return 0;
}

/* SOR with relaxation factor omega (Sec. 2.2, after Eq. 28) for
   (W - h L_W) X = rhs, lexicographic order.  Reading R13: stop when the
   largest update of a sweep is <= sor_tol * max|X|. */
static void sor_rows(const ora_ctx *o, const double *W, double h, const double *rhs,
                     double *X, int r0, int r1, double *maxd, double *maxx);
static int sor(const ora_ctx *o, const double *W, double h, const double *rhs,
               double *X) {
    const int rows = o->D == 2 ? o->p.ny : o->p.nz;
    for (int it = 1; it <= o->p.sor_max_iter; it++) {
        double maxd = 0, maxx = 0;
        sor_rows(o, W, h, rhs, X, 0, rows, &maxd, &maxx);
        if (maxd <= o->p.sor_tol * maxx) return it;
    }
    return -1;
}

int ora_sor(ora_ctx *o, const double *w, double h, const double *rhs,
            double *x) {
    return sor(o, w, h, rhs, x);
}

/* Kahan-compensated FP64 sum (reading R28) */
typedef struct {
    double s, c;
} ksum;
static void kadd(ksum *k, double v) {
    double y = v - k->c;
    double t = k->s + y;
    k->c = (t - k->s) - y;
    k->s = t;
}

/* total surfactant sum (|grad rhoN| + eps) psi + (1 - rhoN + eps) C over the
   grid, with the weights of the current colour field (reading R12, R14) */
static double surf_total(const ora_ctx *o, const double *a, const double *rN,
                         const double *psi, const double *C) {
    ksum k = {0, 0};
    for (long c = 0; c < o->N; c++) {
        kadd(&k, (a[c] + o->p.eps_w) * psi[c]);
        kadd(&k, (1.0 - rN[c] + o->p.eps_w) * C[c]);
    }
    return k.s;
}

/* face neighbours of Eq. 28 (x-, x+, y-, y+, z-, z+); -1 across a wall */
static void build_faces(ora_ctx *o) {
    long N = o->N;
    FOR_CELLS(o) {
        long c = idx(o, x, y, z);
        for (int d = 0; d < o->D; d++)
            for (int s = 0; s < 2; s++) {
                int off[3] = {0, 0, 0}, refl, side[3];
                off[d] = s ? 1 : -1;
                long j = nb(o, x, y, z, off, &refl, side);
                o->face[(2 * d + s) * N + c] = refl ? -1 : j;
            }
    }
}

/* ------------------------------------------------------------------------
 * Context lifecycle
 * ---------------------------------------------------------------------- */
ora_ctx *ora_create(const ora_params *p) {
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return NULL;
    if (p->rhoR0 <= 0 || p->rhoB0 <= 0 || p->muR0 <= 0 || p->muB0 <= 0)
        return NULL;
    ora_ctx *o = (ora_ctx *)calloc(1, sizeof(ora_ctx));
    if (!o) return NULL;
    o->p = *p;
    o->D = p->nz == 1 ? 2 : 3;
    o->N = (long)p->nx * p->ny * p->nz;
    int e[QMAX * 3];
    ora_lattice(o->D, &o->Q, e, o->w, NULL, NULL);
    for (int i = 0; i < o->Q; i++)
        for (int a = 0; a < 3; a++) o->e[i][a] = e[i * 3 + a];
    for (int i = 0; i < o->Q; i++)
        for (int k = 0; k < o->Q; k++)
            if (o->e[k][0] == -o->e[i][0] && o->e[k][1] == -o->e[i][1] &&
                o->e[k][2] == -o->e[i][2])
                o->opp[i] = k;
    for (int m = 0; m < 8; m++)
        for (int i = 0; i < o->Q; i++)
            for (int k = 0; k < o->Q; k++) {
                int same = 1;
                for (int a = 0; a < 3; a++)
                    same &= o->e[k][a] == ((m >> a) & 1 ? -o->e[i][a] : o->e[i][a]);
                if (same) o->mir[m][i] = k;
            }
    long N = o->N, QN = (long)o->Q * N;
    o->fR = calloc(QN, sizeof(double));
    o->fB = calloc(QN, sizeof(double));
    o->fR2 = calloc(QN, sizeof(double));
    o->fB2 = calloc(QN, sizeof(double));
    double **one[] = {&o->psi, &o->C,   &o->Sp,  &o->Bp,  &o->rhoR, &o->rhoB,
                      &o->rho, &o->rhoN, &o->a,  &o->kap, &o->S,    &o->B,
                      &o->rhs, &o->wt,  &o->tmp};
    for (unsigned k = 0; k < sizeof(one) / sizeof(one[0]); k++)
        *one[k] = calloc(N, sizeof(double));
    double **three[] = {&o->g, &o->n, &o->F, &o->u, &o->gpsi, &o->Psi};
    for (unsigned k = 0; k < sizeof(three) / sizeof(three[0]); k++)
        *three[k] = calloc(3 * N, sizeof(double));
    o->face = calloc((size_t)2 * o->D * N, sizeof(long));
    if (!o->fR || !o->fB || !o->fR2 || !o->fB2 || !o->Psi || !o->tmp || !o->face) {
        ora_destroy(o);
        return NULL;
    }
    for (int a = 0; a < 3; a++) o->end[a][0] = o->end[a][1] = p->wall[a];
    build_faces(o);
    return o;
}

/* Boundaries of the two ends of axis a (0 periodic wrap, 1 bounce-back
   wall, 2 mirror plane).  A slab of a decomposed grid wraps at the ends
   where it meets another slab: what the wrap brings into its outermost
   ghost layers is overwritten by the exchange before it can matter. */
int ora_set_ends(ora_ctx *o, int a, int lo, int hi) {
    if (a < 0 || a > 2 || lo < 0 || lo > 2 || hi < 0 || hi > 2) return -1;
    o->end[a][0] = lo;
    o->end[a][1] = hi;
    build_faces(o);
    return 0;
}

void ora_destroy(ora_ctx *o) {
    if (!o) return;
    double *all[] = {o->fR,  o->fB,  o->fR2, o->fB2, o->psi, o->C,   o->Sp,
                     o->Bp,  o->rhoR, o->rhoB, o->rho, o->rhoN, o->a,  o->kap,
                     o->S,   o->B,   o->rhs, o->wt,  o->tmp, o->g,   o->n,
                     o->F,   o->u,   o->gpsi, o->Psi};
    for (unsigned k = 0; k < sizeof(all) / sizeof(all[0]); k++) free(all[k]);
    free(o->face);
    free(o);
}

static void set_M0(ora_ctx *o) {
    macro(o, o->fR, o->fB, o->psi);
    o->M0 = surf_total(o, o->a, o->rhoN, o->psi, o->C);
    o->last_pre = o->M0;
    o->last_scale = 1.0;
}

/* Initial state (reading R20): rho^R = rhoR0 (1+phi)/2, rho^B = rhoB0 (1-phi)/2,
   which reproduces rhoN = phi through Eq. 6, and f^k = M^{-1} m^{k,eq}. */
int ora_init_fields(ora_ctx *o, const double *phi, const double *psi,
                    const double *C, const double *u) {
    long N = o->N;
    double Minv[QMAX * QMAX], mR[QMAX], mB[QMAX];
    ora_lattice(o->D, NULL, NULL, NULL, NULL, Minv);
    for (long c = 0; c < N; c++) {
        double ph = phi[c];
        if (ph > 1.0) ph = 1.0;
        if (ph < -1.0) ph = -1.0;
        double uu[3] = {0, 0, 0};
        if (u)
            for (int a = 0; a < o->D; a++) uu[a] = u[a * N + c];
        ora_meq(o->D, o->p.rhoR0 * 0.5 * (1.0 + ph), uu, o->p.alphaR, mR);
        ora_meq(o->D, o->p.rhoB0 * 0.5 * (1.0 - ph), uu, o->p.alphaB, mB);
        for (int i = 0; i < o->Q; i++) {
            double sr = 0, sb = 0;
            for (int j = 0; j < o->Q; j++) {
                sr += Minv[i * o->Q + j] * mR[j];
                sb += Minv[i * o->Q + j] * mB[j];
            }
            o->fR[i * N + c] = sr;
            o->fB[i * N + c] = sb;
        }
        o->psi[c] = psi ? psi[c] : 0.0;
        o->C[c] = C ? C[c] : 0.0;
        o->Sp[c] = 0.0;
        o->Bp[c] = 0.0;
    }
    o->step = 0;
    o->last_it_psi = o->last_it_C = 0;
    set_M0(o);
    return 0;
}

int ora_set_surfactant(ora_ctx *o, const double *psi, const double *C) {
    memcpy(o->psi, psi, sizeof(double) * o->N);
    memcpy(o->C, C, sizeof(double) * o->N);
    set_M0(o);
    return 0;
}

/* ------------------------------------------------------------------------
 * One coupled time step t -> t+1.  Reading R4 (the paper gives no explicit
 * order): macroscopic fields and forces at t; explicit surfactant terms
 * S^t, B^t; collision, recolouring, streaming; colour weights at t+1;
 * Crank-Nicolson solve for psi, C at t+1; rescaling.
 * ---------------------------------------------------------------------- */
/* steps 1-4: fields and forces at t, explicit terms S^t, B^t, collision,
   recolouring, streaming */
static void phase_lb(ora_ctx *o) {
    const ora_params *p = &o->p;
    long N = o->N;
    int D = o->D, Q = o->Q;

    /* 1. fields at time t: rho^k, rhoN, grad rhoN, kappa, F, u (Eqs. 5-10) */
    macro(o, o->fR, o->fB, o->psi);

    /* 2. explicit terms of Eqs. 23-24 at time t:
          S = -div(psi |grad rhoN| u) + |grad rhoN| j,
          B = -div(C (1 - rhoN) u)    - |grad rhoN| j,
          with j from Eq. 22 (or j = r_a psi_inf C, Sec. 3.1) */
    if (p->transport) {
        for (long c = 0; c < N; c++)
            for (int a = 0; a < 3; a++)
                o->Psi[a * N + c] = o->psi[c] * o->a[c] * o->u[a * N + c];
        weno_div(o, o->Psi, o->u, o->S);
        for (long c = 0; c < N; c++)
            for (int a = 0; a < 3; a++)
                o->Psi[a * N + c] = o->C[c] * (1.0 - o->rhoN[c]) * o->u[a * N + c];
        weno_div(o, o->Psi, o->u, o->B);
        for (long c = 0; c < N; c++) {
            double j = p->source == 1
                           ? p->ra * p->psi_inf * o->C[c]
                           : p->ra * o->C[c] * (p->psi_inf - o->psi[c]) -
                                 p->rd * o->psi[c];
            o->S[c] = -o->S[c] + o->a[c] * j;
            o->B[c] = -o->B[c] - o->a[c] * j;
        }
    }

    /* 3. collision + recolouring at every node (Eqs. 1-4, 11-12) */
    PAR_CELLS(o) {
        long c = idx(o, x, y, z);
        double fr[QMAX], fb[QMAX], fr2[QMAX], fb2[QMAX];
        for (int i = 0; i < Q; i++) {
            fr[i] = o->fR[i * N + c];
            fb[i] = o->fB[i * N + c];
        }
        /* reading R8: d_a(rho^k u_a) by the isotropic derivative at time t;
           rho^k mirrored, u as the ghost velocity at walls */
        double dR[3] = {0, 0, 0}, dB[3] = {0, 0, 0};
        for (int i = 1; i < Q; i++) {
            int refl, side[3];
            long j = nb(o, x, y, z, o->e[i], &refl, side);
            double uj[3];
            ghost_u(o, o->u, j, refl, side, uj);
            for (int a = 0; a < D; a++) {
                dR[a] += o->w[i] * o->rhoR[j] * uj[a] * o->e[i][a];
                dB[a] += o->w[i] * o->rhoB[j] * uj[a] * o->e[i][a];
            }
        }
        for (int a = 0; a < D; a++) {
            dR[a] /= CS2;
            dB[a] /= CS2;
        }
        double uc[3], Fc[3], gc[3];
        for (int a = 0; a < 3; a++) {
            uc[a] = o->u[a * N + c];
            Fc[a] = o->F[a * N + c];
            gc[a] = o->g[a * N + c];
        }
        ora_collide_cell(p, D, fr, fb, uc, Fc, dR, dB, gc, fr2, fb2);
        for (int i = 0; i < Q; i++) {
            o->fR2[i * N + c] = fr2[i];
            o->fB2[i * N + c] = fb2[i];
        }
    }

    /* 4. streaming, Eq. 13, written as a pull: f_i(x, t+1) = f_i^{++}(x - e_i).
          A link that crosses a wall is reflected (half-way bounce-back); a
          moving wall adds 2 w_i rho^k (e_i . u_w)/cs2 (reading R22).  A link
          that crosses only mirror planes brings the mirror image of its
          source: the population of the mirrored direction at the mirrored
          cell (specular reflection). */
    PAR_CELLS(o) {
        long c = idx(o, x, y, z);
        for (int i = 0; i < Q; i++) {
            int back[3] = {-o->e[i][0], -o->e[i][1], -o->e[i][2]};
            int refl, side[3];
            long j = nb(o, x, y, z, back, &refl, side);
            int bbmask = 0; /* axes whose crossing is a bounce-back wall */
            for (int a = 0; a < 3; a++)
                if ((refl & (1 << a)) && o->end[a][side[a] < 0 ? 0 : 1] == 1)
                    bbmask |= 1 << a;
            if (!(refl & bbmask)) {
                int is = o->mir[refl][i];
                o->fR[i * N + c] = o->fR2[is * N + j];
                o->fB[i * N + c] = o->fB2[is * N + j];
                continue;
            }
            double uw[3] = {0, 0, 0};
            int nw = 0;
            for (int a = 0; a < 3; a++) {
                if (!(refl & bbmask & (1 << a))) continue;
                const double *v = side[a] < 0 ? p->uw_lo[a] : p->uw_hi[a];
                for (int b = 0; b < 3; b++) uw[b] += v[b];
                nw++;
            }
            double eu = 0;
            for (int b = 0; b < 3; b++) eu += o->e[i][b] * uw[b] / nw;
            int io = o->opp[i];
            o->fR[i * N + c] = o->fR2[io * N + c] + 2.0 * o->w[i] * o->rhoR[c] * eu / CS2;
            o->fB[i * N + c] = o->fB2[io * N + c] + 2.0 * o->w[i] * o->rhoB[c] * eu / CS2;
        }
    }
}

/* step 5 (transport): the Crank-Nicolson right-hand sides with the
   weights of time t, into rhs (psi) and tmp (C) */
static void phase_rhs(ora_ctx *o) {
    const ora_params *p = &o->p;
    long N = o->N;
    /* 5. Crank-Nicolson right-hand sides with the weights of time t
          (reading R12: a = |grad rhoN| + eps_w, chi = 1 - rhoN + eps_w);
          Euler for the explicit part at t = 0 (Eq. 23), AB2 after (Eq. 24) */
    const double ab_now = o->step == 0 ? 1.0 : 1.5;
    const double ab_old = o->step == 0 ? 0.0 : -0.5;
    double *rhsC = o->tmp;
    for (long c = 0; c < N; c++) o->wt[c] = o->a[c] + p->eps_w;
    diffuse(o, o->wt, o->psi, o->rhs);
    for (long c = 0; c < N; c++)
        o->rhs[c] = o->wt[c] * o->psi[c] + 0.5 * p->Ds * o->rhs[c] +
                    ab_now * o->S[c] + ab_old * o->Sp[c];
    for (long c = 0; c < N; c++) o->wt[c] = 1.0 - o->rhoN[c] + p->eps_w;
    diffuse(o, o->wt, o->C, rhsC);
    for (long c = 0; c < N; c++)
        rhsC[c] = o->wt[c] * o->C[c] + 0.5 * p->Db * rhsC[c] +
                  ab_now * o->B[c] + ab_old * o->Bp[c];
}

/* one lexicographic SOR sweep (Sec. 2.2) over the rows [r0, r1) of the
   slowest axis (y in 2D, z in 3D) for (W - h L_W) X = rhs; folds the largest
   update and the largest |X| of the sweep into *maxd, *maxx */
static void sor_rows(const ora_ctx *o, const double *W, double h, const double *rhs,
                     double *X, int r0, int r1, double *maxd, double *maxx) {
    const double om = o->p.sor_omega;
    const long row = o->N / (o->D == 2 ? o->p.ny : o->p.nz);
    for (long c = r0 * row; c < r1 * row; c++) { /* lexicographic: x fastest */
        double diag = W[c], off = 0;
        for (int f = 0; f < 2 * o->D; f++) {
            long j = o->face[f * o->N + c];
            if (j < 0) continue;
            double wf = 0.5 * (W[c] + W[j]);
            diag += h * wf;
            off += h * wf * X[j];
        }
        double xn = (rhs[c] + off) / diag;
        double dx = om * (xn - X[c]);
        X[c] += dx;
        if (fabs(dx) > *maxd) *maxd = fabs(dx);
        if (fabs(X[c]) > *maxx) *maxx = fabs(X[c]);
    }
}

/* step 8 after the solves: rescale by s, keep the explicit terms as the
   Adams-Bashforth history, count the step */
static void phase_finish(ora_ctx *o, double s, double pre) {
    long N = o->N;
    if (o->p.transport) {
        for (long c = 0; c < N; c++) {
            o->psi[c] *= s;
            o->C[c] *= s;
        }
        o->last_pre = pre;
        o->last_scale = s;
        memcpy(o->Sp, o->S, sizeof(double) * N);
        memcpy(o->Bp, o->B, sizeof(double) * N);
    }
    o->step++;
}

static int one_step(ora_ctx *o) {
    const ora_params *p = &o->p;
    long N = o->N;
    phase_lb(o);
    if (!p->transport) {
        phase_finish(o, 1.0, 0.0);
        return 0;
    }
    phase_rhs(o);
    double *rhsC = o->tmp;

    /* 6. weights at t+1 from the streamed populations */
    macro(o, o->fR, o->fB, o->psi);

    /* 7. implicit solves (W^{t+1} - (D/2) L_{W^{t+1}}) X^{t+1} = rhs by SOR */
    for (long c = 0; c < N; c++) o->wt[c] = o->a[c] + p->eps_w;
    int itp = sor(o, o->wt, 0.5 * p->Ds, o->rhs, o->psi);
    for (long c = 0; c < N; c++) o->wt[c] = 1.0 - o->rhoN[c] + p->eps_w;
    int itc = sor(o, o->wt, 0.5 * p->Db, rhsC, o->C);
    o->last_it_psi = itp;
    o->last_it_C = itc;
    if (itp < 0 || itc < 0) return -4;

    /* 8. rescale psi and C by one common factor so that the total
          surfactant equals its initial value (reading R14) */
    double Mt = surf_total(o, o->a, o->rhoN, o->psi, o->C);
    phase_finish(o, Mt > 0 ? o->M0 / Mt : 1.0, Mt);
    return 0;
}

/* ---- building blocks of a step, for a grid decomposed into slabs ---- */

int ora_phase(ora_ctx *o, int k) {
    const ora_params *p = &o->p;
    long N = o->N;
    switch (k) {
    case 0: phase_lb(o); return 0;
    case 1: phase_rhs(o); return 0;
    case 2: macro(o, o->fR, o->fB, o->psi); return 0;
    case 3:
        for (long c = 0; c < N; c++) o->wt[c] = o->a[c] + p->eps_w;
        return 0;
    case 4:
        for (long c = 0; c < N; c++) o->wt[c] = 1.0 - o->rhoN[c] + p->eps_w;
        return 0;
    }
    return -1;
}

int ora_sor_rows(ora_ctx *o, int which, int r0, int r1, double *maxd, double *maxx) {
    if (which == 0)
        sor_rows(o, o->wt, 0.5 * o->p.Ds, o->rhs, o->psi, r0, r1, maxd, maxx);
    else
        sor_rows(o, o->wt, 0.5 * o->p.Db, o->tmp, o->C, r0, r1, maxd, maxx);
    return 0;
}

int ora_surf_rows(ora_ctx *o, int r0, int r1, double *ks) {
    const long row = o->N / (o->D == 2 ? o->p.ny : o->p.nz);
    ksum k = {ks[0], ks[1]};
    for (long c = r0 * row; c < r1 * row; c++) {
        kadd(&k, (o->a[c] + o->p.eps_w) * o->psi[c]);
        kadd(&k, (1.0 - o->rhoN[c] + o->p.eps_w) * o->C[c]);
    }
    ks[0] = k.s;
    ks[1] = k.c;
    return 0;
}

int ora_finish(ora_ctx *o, double s, double pre, int itp, int itc) {
    o->last_it_psi = itp;
    o->last_it_C = itc;
    phase_finish(o, s, pre);
    return 0;
}

void ora_set_M0(ora_ctx *o, double M0) {
    o->M0 = M0;
    o->last_pre = M0;
}

double *ora_field(ora_ctx *o, const char *name) {
    struct {
        const char *n;
        double *p;
    } t[] = {{"fR", o->fR}, {"fB", o->fB}, {"psi", o->psi}, {"C", o->C}, {"Sp", o->Sp},
             {"Bp", o->Bp}, {"a", o->a},   {"rhoN", o->rhoN}};
    for (unsigned k = 0; k < sizeof(t) / sizeof(t[0]); k++)
        if (!strcmp(t[k].n, name)) return t[k].p;
    return NULL;
}

int ora_step(ora_ctx *o, int n) {
    for (int k = 0; k < n; k++) {
        int r = one_step(o);
        if (r) return r;
    }
    return 0;
}

long long ora_step_count(const ora_ctx *o) { return o->step; }

#ifdef _OPENMP
#include <omp.h>
#endif
/* host threads the cell loops use (1 without OpenMP); n <= 0 leaves it */
int ora_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

int ora_macro(ora_ctx *o, double *rhoR, double *rhoB, double *rhoN, double *g,
              double *a, double *kappa, double *F, double *u, double *S,
              double *B) {
    long N = o->N;
    macro(o, o->fR, o->fB, o->psi);
    if (S || B) {
        /* the explicit terms as computed in step 2 of one_step */
        for (long c = 0; c < N; c++)
            for (int d = 0; d < 3; d++)
                o->Psi[d * N + c] = o->psi[c] * o->a[c] * o->u[d * N + c];
        weno_div(o, o->Psi, o->u, o->S);
        for (long c = 0; c < N; c++)
            for (int d = 0; d < 3; d++)
                o->Psi[d * N + c] = o->C[c] * (1.0 - o->rhoN[c]) * o->u[d * N + c];
        weno_div(o, o->Psi, o->u, o->B);
        const ora_params *p = &o->p;
        for (long c = 0; c < N; c++) {
            double j = p->source == 1
                           ? p->ra * p->psi_inf * o->C[c]
                           : p->ra * o->C[c] * (p->psi_inf - o->psi[c]) -
                                 p->rd * o->psi[c];
            if (S) S[c] = -o->S[c] + o->a[c] * j;
            if (B) B[c] = -o->B[c] - o->a[c] * j;
        }
    }
    if (rhoR) memcpy(rhoR, o->rhoR, sizeof(double) * N);
    if (rhoB) memcpy(rhoB, o->rhoB, sizeof(double) * N);
    if (rhoN) memcpy(rhoN, o->rhoN, sizeof(double) * N);
    if (g) memcpy(g, o->g, sizeof(double) * 3 * N);
    if (a) memcpy(a, o->a, sizeof(double) * N);
    if (kappa) memcpy(kappa, o->kap, sizeof(double) * N);
    if (F) memcpy(F, o->F, sizeof(double) * 3 * N);
    if (u) memcpy(u, o->u, sizeof(double) * 3 * N);
    return 0;
}

int ora_get_fields(ora_ctx *o, double *rho, double *u, double *phi,
                   double *psi, double *C) {
    long N = o->N;
    macro(o, o->fR, o->fB, o->psi);
    if (rho) memcpy(rho, o->rho, sizeof(double) * N);
    if (u) memcpy(u, o->u, sizeof(double) * 3 * N);
    if (phi) memcpy(phi, o->rhoN, sizeof(double) * N);
    if (psi) memcpy(psi, o->psi, sizeof(double) * N);
    if (C) memcpy(C, o->C, sizeof(double) * N);
    return 0;
}

int ora_get_pops(ora_ctx *o, double *fR, double *fB) {
    size_t b = sizeof(double) * (size_t)o->Q * o->N;
    if (fR) memcpy(fR, o->fR, b);
    if (fB) memcpy(fB, o->fB, b);
    return 0;
}

int ora_set_pops(ora_ctx *o, const double *fR, const double *fB) {
    size_t b = sizeof(double) * (size_t)o->Q * o->N;
    memcpy(o->fR, fR, b);
    memcpy(o->fB, fB, b);
    return 0;
}

/* Diagnostics: droplet velocity U of Eqs. 33-34 (mean velocity over the
   nodes with rhoN >= 0), centroid, aspect ratio from the second moments of
   that indicator, Re = 2 rhoB0 U R / muB0 (Sec. 3.4), interface psi
   statistics, conservation totals. */
int ora_diagnostics(ora_ctx *o, ora_diag *d) {
    const ora_params *p = &o->p;
    long N = o->N;
    macro(o, o->fR, o->fB, o->psi);
    memset(d, 0, sizeof(*d));
    ksum mR = {0, 0}, mB = {0, 0};
    double cnt = 0, su[3] = {0, 0, 0}, sx[3] = {0, 0, 0};
    double pav = 0, pcnt = 0, pmin = HUGE_VAL, pmax = -HUGE_VAL, umax = 0;
    /* vertical axis: the axis of gravity, else the last axis */
    int vert = o->D - 1;
    double gmax = 0;
    for (int a = 0; a < o->D; a++)
        if (fabs(p->g[a]) > gmax) {
            gmax = fabs(p->g[a]);
            vert = a;
        }
    FOR_CELLS(o) {
        long c = idx(o, x, y, z);
        kadd(&mR, o->rhoR[c]);
        kadd(&mB, o->rhoB[c]);
        double um = 0;
        for (int a = 0; a < 3; a++) um += o->u[a * N + c] * o->u[a * N + c];
        if (sqrt(um) > umax) umax = sqrt(um);
        if (o->rhoN[c] >= 0.0) {
            int xyz[3] = {x, y, z};
            cnt += 1;
            for (int a = 0; a < 3; a++) {
                su[a] += o->u[a * N + c];
                sx[a] += xyz[a];
            }
        }
        if (fabs(o->rhoN[c]) < 0.5) {
            pav += o->psi[c];
            pcnt += 1;
            if (o->psi[c] < pmin) pmin = o->psi[c];
            if (o->psi[c] > pmax) pmax = o->psi[c];
        }
    }
    d->mass_R = mR.s;
    d->mass_B = mB.s;
    d->surf_total = surf_total(o, o->a, o->rhoN, o->psi, o->C);
    d->surf_pre_rescale = o->last_pre;
    d->rescale_factor = o->last_scale;
    if (cnt > 0) {
        for (int a = 0; a < 3; a++) {
            d->U[a] = su[a] / cnt;
            d->centroid[a] = sx[a] / cnt;
        }
        double I[3] = {0, 0, 0};
        FOR_CELLS(o) {
            long c = idx(o, x, y, z);
            if (o->rhoN[c] < 0.0) continue;
            int xyz[3] = {x, y, z};
            for (int a = 0; a < 3; a++)
                I[a] += (xyz[a] - d->centroid[a]) * (xyz[a] - d->centroid[a]);
        }
        int hor = vert == 0 ? 1 : 0;
        d->aspect_ratio = I[vert] > 0 ? sqrt(I[hor] / I[vert]) : 0.0;
        double R = o->D == 2 ? sqrt(cnt / M_PI) : cbrt(3.0 * cnt / (4.0 * M_PI));
        d->Re = 2.0 * p->rhoB0 * fabs(d->U[vert]) * R / p->muB0;
    }
    if (pcnt > 0) {
        d->psi_av = pav / pcnt;
        d->psi_min = pmin;
        d->psi_max = pmax;
    }
    d->umax = umax;
    d->sor_iters_psi = o->last_it_psi;
    d->sor_iters_C = o->last_it_C;
    d->step = o->step;
    return 0;
}
