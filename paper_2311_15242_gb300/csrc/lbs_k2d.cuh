// lbs_k2d.cuh — D2Q9 kernels of the coupled LB-FD time step (arXiv 2311.15242).
//
// Storage form of the populations.  For every cell and direction the library
// keeps fT_i = f_i - s_i, the total f_i = f_i^R + f_i^B minus a constant rest
// state s_i (the rest equilibrium of the pure blue phase; for the alpha-model
// of App. A both pure phases share its moving components), and fM_i, the
// population of the cell's minority colour (a per-cell flag says which).  The
// majority colour is s_i + fT_i - fM_i.  Momentum and every non-conserved
// moment are formed from small numbers, and the colour that is nearly absent
// keeps its full relative precision; both matter in FP32: the interface
// weights |grad rho^N| and 1 - rho^N of the surfactant equations are divided
// by a regularisation of 1e-6 where they vanish.
//
// One time step (t -> t+1) is the kernel sequence
//   k_force    u, F at t                   (Eqs. 5-10)
//   k_fd       S^t, B^t, CN right-hand sides (Eqs. 22-28)
//   k_collide  collision + recolouring      (Eqs. 1-4, 11-12, App. A)
//   k_stream   streaming, bounce-back, moments at t+1 (Eq. 13)
//   k_grad     grad rhoN, |grad rhoN|, 1 - rhoN at t+1
//   k_sor      red-black SOR sweeps        (Sec. 2.2)
//   k_surf     total surfactant, rescale factor (Sec. 2.2)
//   k_scale    psi, C *= factor
#pragma once

#include "lbs_dev.cuh"

namespace lbs {

template <typename R>
__device__ __forceinline__ R cs2_lattice() { return R(1) / R(3); }

// shift of direction i for a cell with the given flag
template <typename R>
__device__ __forceinline__ R shift_of(const Inst<R> &I, int i, int flag) {
    return i == 0 ? I.shift0[flag] : I.shift[i];
}


// colour densities and momentum (without the force) of one cell
template <typename R>
struct Mom2 {
    R rR, rB, drho, jx, jy;  // rho^R, rho^B, rho - rho_s[flag], sum_i f_i e_i
    R rm_s, rm_c, dr_s, dr_c;  // minority mass and drho as unevaluated sums s + c
};

// compensated summation (Knuth's TwoSum): s + c carries the sum of the added
// terms to about twice the working precision.  The colour masses of the
// recolouring split are formed this way: a plainly rounded sum of nine
// similar terms has nearly the same rounding error in neighbouring cells,
// which biases the colour mass the same way every step.
template <typename R>
struct CSum {
    R s = R(0), c = R(0);
    __device__ __forceinline__ void add(R v) {
        R t = s + v;
        R bp = t - s;
        c += (s - (t - bp)) + (v - bp);
        s = t;
    }
    __device__ __forceinline__ R value() const { return s + c; }
};

template <typename R>
__device__ __forceinline__ Mom2<R> moments9(const Inst<R> &I, const R *fT, const R *fM,
                                           int flag) {
    Mom2<R> m{R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0)};
    CSum<R> rmc, drc;
#pragma unroll
    for (int i = 0; i < Q9; i++) {
        rmc.add(fM[i]);
        drc.add(fT[i]);
        m.jx += R(ex9(i)) * fT[i];
        m.jy += R(ey9(i)) * fT[i];
    }
    const R rm = rmc.value();
    m.drho = drc.value();
    m.rm_s = rmc.s;
    m.rm_c = rmc.c;
    m.dr_s = drc.s;
    m.dr_c = drc.c;
    // majority colour = total - minority
    R rmaj = (I.rho_s[flag] - rm) + m.drho;
    m.rR = flag ? rmaj : rm;
    m.rB = flag ? rm : rmaj;
    return m;
}

// minority colour of a cell by colour fraction (0: red, 1: blue)
template <typename R>
__device__ __forceinline__ int minority(const Inst<R> &I, R rR, R rB) {
    return (rR * I.inv_rhoR0 <= rB * I.inv_rhoB0) ? 0 : 1;
}

// colour function, Eq. 6
template <typename R>
__device__ __forceinline__ R colour_fn(const Inst<R> &I, R rR, R rB) {
    const R xr = rR * I.inv_rhoR0, xb = rB * I.inv_rhoB0;
    return fdiv(xr - xb, xr + xb);
}

// ---------------------------------------------------------------------------
// Initial populations: f^k = M^{-1} m^{k,eq}(rho^k, u) (App. A), rho^R and
// rho^B from the colour field.  Inputs are dense double arrays [ny][nx].
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ void meq9(R rho, R ux, R uy, R al, R *m) {
    R u2 = ux * ux + uy * uy;
    m[0] = rho;
    m[1] = rho * (R(-3.6) * al - R(0.4) + R(3) * u2);
    m[2] = rho * (R(5.4) * al - R(1.4) - R(3) * u2);
    m[3] = rho * ux;
    m[4] = rho * (R(-1.8) * al - R(0.2)) * ux;
    m[5] = rho * uy;
    m[6] = rho * (R(-1.8) * al - R(0.2)) * uy;
    m[7] = rho * (ux * ux - uy * uy);
    m[8] = rho * ux * uy;
}

// f = M^{-1} m = M^T diag(1 / |row j|^2) m.  Each moment is divided by its
// row norm once; the entries of M are 0, +-1, +-2 or +-4, so a (m_j / n_j)
// equals (a m_j) / n_j exactly (nine divisions instead of one a term: this
// runs in FP64, on GB300's narrow FP64 pipe)
template <typename R>
__device__ __forceinline__ void minv9(const R *m, R *f) {
    R mn[Q9];
#pragma unroll
    for (int j = 0; j < Q9; j++) mn[j] = m[j] / R(mnorm9(j));
#pragma unroll
    for (int i = 0; i < Q9; i++) {
        R s = R(0);
#pragma unroll
        for (int j = 0; j < Q9; j++)
            if (m9(j, i) != 0) s += R(m9(j, i)) * mn[j];
        f[i] = s;
    }
}

template <typename R, typename P>
__global__ void k_init2(Inst<R> I, const double *phi, const double *psi, const double *C,
                        const double *u) {
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= I.nx || y >= I.ny) return;
    long long d = (long long)y * I.nx + x;
    long long c = (long long)y * I.pitch + x;
    long long N = (long long)I.nx * I.ny;
    double ph = phi[d];
    ph = ph > 1.0 ? 1.0 : (ph < -1.0 ? -1.0 : ph);
    // built in double precision and rounded once, so that the stored
    // deviations carry no direction-dependent rounding of the equilibrium
    double ux = u ? u[d] : 0.0, uy = u ? u[N + d] : 0.0;
    double mR[Q9], mB[Q9], fR[Q9], fB[Q9];
    const double rR = double(I.rhoR0) * 0.5 * (1.0 + ph), rB = double(I.rhoB0) * 0.5 * (1.0 - ph);
    meq9<double>(rR, ux, uy, double(I.alphaR), mR);
    meq9<double>(rB, ux, uy, double(I.alphaB), mB);
    minv9<double>(mR, fR);
    minv9<double>(mB, fB);
    const int fl = (rR / double(I.rhoR0) <= rB / double(I.rhoB0)) ? 0 : 1;
    // moving populations rounded to the storage type; the rest populations
    // take what the rounding left out, so the stored masses are the intended ones
    double tT = 0, tM = 0, sT = 0, sM = 0;
#pragma unroll
    for (int i = 0; i < Q9; i++) {
        const double vT = (fR[i] + fB[i]) - double(shift_of(I, i, fl)), vM = fl ? fB[i] : fR[i];
        tT += vT;
        tM += vM;
        if (i) {
            sT += double(stq<R, P>(I, I.fT, i, c, R(vT)));
            sM += double(stq<R, P>(I, I.fM, i, c, R(vM)));
        }
    }
    I.fT0[c] = R(tT - sT);
    I.fM0[c] = R(tM - sM);
    I.flag[c] = (uint8_t)fl;
    I.psi[c] = psi ? R(psi[d]) : R(0);
    I.C[c] = C ? R(C[d]) : R(0);
    I.psip[c] = I.psi[c];
    I.Cp[c] = I.C[c];
    I.S[c] = R(0);
    I.B[c] = R(0);
}

// initial guess of the Crank-Nicolson solves (Sec. 2.2): the linear
// extrapolation 2 x^n - x^(n-1) of the last two time levels instead of
// x^n; SOR converges to the same solution within its tolerance in fewer
// sweeps.  Elementwise (run where no kernel reads psi, C of neighbours).
template <typename R>
__device__ __forceinline__ void sor_guess(const Inst<R> &I, long long c) {
    if (!I.transport) return;
    const R p = I.psi[c], q = I.C[c];
    I.psi[c] = R(2) * p - I.psip[c];
    I.C[c] = R(2) * q - I.Cp[c];
    I.psip[c] = p;
    I.Cp[c] = q;
}

// moments of the stored populations -> rho^R, rho^B, rho^N, momentum
template <typename R>
__device__ __forceinline__ void store_moments(const Inst<R> &I, long long c, const R *fT,
                                              const R *fM, int flag) {
    Mom2<R> m = moments9(I, fT, fM, flag);
    I.rhoR[c] = m.rR;
    I.rhoB[c] = m.rB;
    I.rhoN[c] = colour_fn(I, m.rR, m.rB);
    I.jx[c] = m.jx;
    I.jy[c] = m.jy;
}

template <typename R, typename P>
__global__ void k_moments2(Inst<R> I) {
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= I.nx || y >= I.ny) return;
    long long c = (long long)y * I.pitch + x;
    R fT[Q9], fM[Q9];
#pragma unroll
    for (int i = 0; i < Q9; i++) {
        fT[i] = ldq<R, P>(I, I.fT, I.fT0, i, c);
        fM[i] = ldq<R, P>(I, I.fM, I.fM0, i, c);
    }
    store_moments(I, c, fT, fM, I.flag[c]);
}

// ---------------------------------------------------------------------------
// k_grad: colour gradient by the isotropic stencil (Sec. 2.1 after Eq. 9):
// d_a X = (1/c_s^2) sum_i w_i X(x + e_i) e_ia, rho^N mirrored at walls;
// a = |grad rho^N| and chi = 1 - rho^N.  Since rho^N = 2 phi_R - 1 = 1 - 2 phi_B
// with the colour fractions phi_k = x_k / (x_R + x_B), x_k = rho^k / rho^k0,
// the gradient is taken as 2 grad phi_R on the blue side and -2 grad phi_B on
// the red side (the same number, formed from the colour that is small there),
// and chi = 2 phi_B.
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ R frac_of(const Inst<R> &I, const R *rR, const R *rB, long long j,
                                     bool red) {
    const R xr = rR[j] * I.inv_rhoR0, xb = rB[j] * I.inv_rhoB0;
    return fdiv(red ? xr : xb, xr + xb);
}
template <typename R>
__device__ __forceinline__ R frac(const Inst<R> &I, long long j, bool red) {
    return frac_of(I, I.rhoR, I.rhoB, j, red);
}

// gradient and weights of cell (x, y) from the colour densities rR, rB and
// colour function rN (the current moments, or the next ones of the fused step)
template <typename R>
__device__ __forceinline__ void grad2_cell_from(const Inst<R> &I, int x, int y, const R *rR,
                                                const R *rB, const R *rN) {
    long long c = (long long)y * I.pitch + x;
    const bool blue_side = rN[c] <= R(0);
    const Ax X = make_ax(x, I.nx, I.wall[0], 1), Y = make_ax(y, I.ny, I.wall[1], 2);
    R gx = R(0), gy = R(0);
#pragma unroll
    for (int i = 1; i < Q9; i++) {
        int refl, sx, sy;
        long long j = nbx2(I, X, Y, ex9(i), ey9(i), refl, sx, sy);
        R v = frac_of(I, rR, rB, j, blue_side);
        gx += w9<R>(i) * R(ex9(i)) * v;
        gy += w9<R>(i) * R(ey9(i)) * v;
    }
    const R f = blue_side ? R(6) : R(-6);  // 2 / c_s^2
    gx *= f;
    gy *= f;
    I.gx[c] = gx;
    I.gy[c] = gy;
    I.a[c] = sqrt(gx * gx + gy * gy);
    I.chi[c] = R(2) * frac_of(I, rR, rB, c, false);
}

template <typename R>
__device__ __forceinline__ void grad2_cell(const Inst<R> &I, int x, int y, bool guess = true) {
    if (x >= I.nx || y >= I.ny) return;
    grad2_cell_from(I, x, y, I.rhoR, I.rhoB, I.rhoN);
    if (guess) sor_guess(I, (long long)y * I.pitch + x);
}

// guess: also form the SOR initial guess (every step; not at initialisation).
// The kernel runs just before the one-launch SOR of the step, so it also
// clears that launch's grid-barrier arrival counter: a barrier that gave up
// (ST_TIMEOUT) leaves a partial count behind, which would release the next
// launch's first barrier early.
template <typename R>
__global__ void k_grad2(Inst<R> I, int guess = 1) {
    pdl_wait();
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && threadIdx.y == 0)
        I.ctl->bar_count = 0;
    grad2_cell(I, blockIdx.x * blockDim.x + threadIdx.x, blockIdx.y * blockDim.y + threadIdx.y,
               guess != 0);
}

// ---------------------------------------------------------------------------
// k_force: n = -grad rhoN / |grad rhoN| (regularised by eps_n), curvature
// kappa = -div n (Eq. 7), grad psi, sigma(psi) (Eq. 8), interfacial force
// (Eq. 9) plus buoyancy (rho - rhoB0) g (Sec. 3.4), velocity of Eq. 10.
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ void force2_cell(const Inst<R> &I, int x, int y) {
    if (x >= I.nx || y >= I.ny) return;
    long long c = (long long)y * I.pitch + x;
    const R e2 = I.eps_n * I.eps_n;
    const Ax X = make_ax(x, I.nx, I.wall[0], 1), Y = make_ax(y, I.ny, I.wall[1], 2);
    R divn = R(0), dpx = R(0), dpy = R(0);
#pragma unroll
    for (int i = 1; i < Q9; i++) {
        int refl, sx, sy;
        long long j = nbx2(I, X, Y, ex9(i), ey9(i), refl, sx, sy);
        R gx = I.gx[j], gy = I.gy[j];
        if (refl & 1) gx = -gx;  // normal component mirrored with a sign change
        if (refl & 2) gy = -gy;
        R inv = frsq(gx * gx + gy * gy + e2);
        R nx = -gx * inv, ny = -gy * inv;
        divn += w9<R>(i) * (R(ex9(i)) * nx + R(ey9(i)) * ny);
        R p = I.psi[j];
        dpx += w9<R>(i) * R(ex9(i)) * p;
        dpy += w9<R>(i) * R(ey9(i)) * p;
    }
    R kappa = -R(3) * divn;
    dpx *= R(3);
    dpy *= R(3);
    R gx = I.gx[c], gy = I.gy[c], a = I.a[c];
    R sigma, mco;
    R Fx, Fy;
    if (eos(I, I.psi[c], sigma, mco)) {
        R inv = frsq(gx * gx + gy * gy + e2);
        R nx = -gx * inv, ny = -gy * inv;
        R ndp = nx * dpx + ny * dpy;
        Fx = -R(0.5) * sigma * kappa * gx - R(0.5) * a * mco * (dpx - ndp * nx);
        Fy = -R(0.5) * sigma * kappa * gy - R(0.5) * a * mco * (dpy - ndp * ny);
    } else {
        Fx = -R(0.5) * I.sigma_min * kappa * gx;
        Fy = -R(0.5) * I.sigma_min * kappa * gy;
    }
    // (the moments of the current step: set 0 but in the fused step's form)
    const MomSet<R> m = mom_of_step(I, I.ctl->step);
    R rR = m.rR[c], rB = m.rB[c];
    R rho = rR + rB;
    // (rho - rhoB0) = rho^R + (rho^B - rhoB0)
    R drb = rR + (rB - I.rhoB0);
    Fx += drb * I.g[0];
    Fy += drb * I.g[1];
    I.Fx[c] = Fx;
    I.Fy[c] = Fy;
    const R irho = fdiv(R(1), rho);
    I.ux[c] = (m.jx[c] + R(0.5) * Fx) * irho;
    I.uy[c] = (m.jy[c] + R(0.5) * Fy) * irho;
}

template <typename R>
__global__ void k_force2(Inst<R> I) {
    pdl_trigger();
    force2_cell(I, blockIdx.x * blockDim.x + threadIdx.x, blockIdx.y * blockDim.y + threadIdx.y);
}

// ---------------------------------------------------------------------------
// k_fd: explicit terms of Eqs. 23-24 at time t and the Crank-Nicolson
// right-hand sides.
//   S = -div(psi a u) + a j,  B = -div(C chi u) - a j   (Eq. 22 for j)
//   div by the WENO3 one-sided differences of Eqs. 25-27, upwinded by the sign
//   of the local velocity component (mean of both sides where it is zero)
//   rhs_psi = w psi + (Ds/2) L_w psi + {S (t = 0) | 3/2 S - 1/2 S_prev}
//   with w = a + eps_w and L_w the flux-form operator of Eq. 28.
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ R weno_m(const R *v) {  // v points at node i, v[-2..1]
    const R eps = R(1e-6);
    R d2m = v[0] - R(2) * v[-1] + v[-2];
    R d20 = v[1] - R(2) * v[0] + v[-1];
    R r = fdiv(eps + d2m * d2m, eps + d20 * d20);
    R w = fdiv(R(1), R(1) + R(2) * r * r);
    R dpm2 = v[-1] - v[-2], dpm1 = v[0] - v[-1], dp0 = v[1] - v[0];
    return R(0.5) * ((dpm1 + dp0) - w * (dpm2 - R(2) * dpm1 + dp0));
}
template <typename R>
__device__ __forceinline__ R weno_p(const R *v) {  // v[-1..2]
    const R eps = R(1e-6);
    R d2p = v[2] - R(2) * v[1] + v[0];
    R d20 = v[1] - R(2) * v[0] + v[-1];
    R r = fdiv(eps + d2p * d2p, eps + d20 * d20);
    R w = fdiv(R(1), R(1) + R(2) * r * r);
    R dpm1 = v[0] - v[-1], dp0 = v[1] - v[0], dp1 = v[2] - v[1];
    return R(0.5) * ((dpm1 + dp0) - w * (dp1 - R(2) * dp0 + dpm1));
}
template <typename R>
__device__ __forceinline__ R upwind(const R *v, R u) {
    if (u > R(0)) return weno_m(v);
    if (u < R(0)) return weno_p(v);
    return R(0.5) * (weno_m(v) + weno_p(v));
}

// Sout, Bout: when given, only S and B of the current state are written
// there (export; the Adams-Bashforth history and the right-hand sides are
// left untouched)
template <typename R>
__device__ __forceinline__ void fd2_cell(const Inst<R> &I, int x, int y, double *Sout,
                                         double *Bout) {
    if (x >= I.nx || y >= I.ny) return;
    long long c = (long long)y * I.pitch + x;
    // line values of Psi_x, Phi_x along x and Psi_y, Phi_y along y
    R Px[5], Cx[5], Py[5], Cy[5];
    const Ax X = make_ax(x, I.nx, I.wall[0], 1), Y = make_ax(y, I.ny, I.wall[1], 2);
#pragma unroll
    for (int k = -2; k <= 2; k++) {
        int refl, sx, sy;
        long long j = nbx2(I, X, Y, k, 0, refl, sx, sy);
        R sgn = (refl & 1) ? R(-1) : R(1);
        R u = I.ux[j];
        Px[k + 2] = sgn * I.psi[j] * I.a[j] * u;
        Cx[k + 2] = sgn * I.C[j] * I.chi[j] * u;
        j = nbx2(I, X, Y, 0, k, refl, sx, sy);
        sgn = (refl & 2) ? R(-1) : R(1);
        u = I.uy[j];
        Py[k + 2] = sgn * I.psi[j] * I.a[j] * u;
        Cy[k + 2] = sgn * I.C[j] * I.chi[j] * u;
    }
    R ux = I.ux[c], uy = I.uy[c];
    R divP = upwind(Px + 2, ux) + upwind(Py + 2, uy);
    R divC = upwind(Cx + 2, ux) + upwind(Cy + 2, uy);
    R psi = I.psi[c], Cc = I.C[c], a = I.a[c];
    R j = I.source == 1 ? I.ra * I.psi_inf * Cc
                        : I.ra * Cc * (I.psi_inf - psi) - I.rd * psi;
    R S = -divP + a * j;
    R B = -divC - a * j;
    if (Sout) {
        long long d = (long long)y * I.nx + x;
        Sout[d] = S;
        Bout[d] = B;
        return;
    }
    // diffusion operator of Eq. 28 with the weights of time t
    R wp = a + I.eps_w, wc = I.chi[c] + I.eps_w;
    R Lp = R(0), Lc = R(0);
#pragma unroll
    for (int f = 0; f < 4; f++) {
        int dx = f == 0 ? -1 : (f == 1 ? 1 : 0);
        int dy = f == 2 ? -1 : (f == 3 ? 1 : 0);
        int refl, sx, sy;
        long long j2 = nbx2(I, X, Y, dx, dy, refl, sx, sy);
        if (refl) continue;
        Lp += R(0.5) * (wp + (I.a[j2] + I.eps_w)) * (I.psi[j2] - psi);
        Lc += R(0.5) * (wc + (I.chi[j2] + I.eps_w)) * (I.C[j2] - Cc);
    }
    const bool first = I.ctl->step == 0;
    R Sp = I.S[c], Bp = I.B[c];
    R abS = first ? S : R(1.5) * S - R(0.5) * Sp;
    R abB = first ? B : R(1.5) * B - R(0.5) * Bp;
    I.rpsi[c] = wp * psi + R(0.5) * I.Ds * Lp + abS;
    I.rC[c] = wc * Cc + R(0.5) * I.Db * Lc + abB;
    I.S[c] = S;
    I.B[c] = B;
}

template <typename R>
__global__ void k_fd2(Inst<R> I, double *Sout = nullptr, double *Bout = nullptr) {
    fd2_cell(I, blockIdx.x * blockDim.x + threadIdx.x, blockIdx.y * blockDim.y + threadIdx.y, Sout, Bout);
}

// ---------------------------------------------------------------------------
// k_collide: MRT collision with correction and forcing in moment space
// (Eqs. 1-4, App. A Eqs. 36-38, 43) on the total populations, then
// recolouring (Eqs. 11-12).  Output: post-collision buffers gT, gR.
// ---------------------------------------------------------------------------
template <typename R, typename P>
__device__ __forceinline__ void collide2_cell(const Inst<R> &I, int x, int y) {
    if (x >= I.nx || y >= I.ny) return;
    long long c = (long long)y * I.pitch + x;
    R fT[Q9], fM[Q9];
    const int fl = I.flag[c];
#pragma unroll
    for (int i = 0; i < Q9; i++) {
        fT[i] = ldq<R, P>(I, I.fT, I.fT0, i, c);
        fM[i] = ldq<R, P>(I, I.fM, I.fM0, i, c);
    }
    Mom2<R> mo = moments9(I, fT, fM, fl);
    const R rR = mo.rR, rB = mo.rB;
    const R rmin = fl ? rB : rR;
    // deviation of the majority colour from its pure-phase density
    const R devmaj = I.dsh[fl] + (mo.drho - rmin);
    const R rho = rR + rB;
    const R ux = I.ux[c], uy = I.uy[c], Fx = I.Fx[c], Fy = I.Fy[c];

    // d_a(rho^k u_a) by the isotropic stencil, u at walls as the ghost velocity
    R dRx = R(0), dRy = R(0), dBx = R(0), dBy = R(0);
    const Ax X = make_ax(x, I.nx, I.wall[0], 1), Y = make_ax(y, I.ny, I.wall[1], 2);
#pragma unroll
    for (int i = 1; i < Q9; i++) {
        int refl, sx, sy;
        long long j = nbx2(I, X, Y, ex9(i), ey9(i), refl, sx, sy);
        R vx = I.ux[j], vy = I.uy[j];
        ghost_u2(I, refl, sx, sy, vx, vy);
        R r1 = I.rhoR[j], r2 = I.rhoB[j];
        R wx = w9<R>(i) * R(ex9(i)), wy = w9<R>(i) * R(ey9(i));
        dRx += wx * r1 * vx;
        dRy += wy * r1 * vy;
        dBx += wx * r2 * vx;
        dBy += wy * r2 * vy;
    }
    // Q^k = (1.8 alpha^k - 0.8) d(rho^k u); correction C (Eq. 37), summed over k
    const R cR = R(1.8) * I.alphaR - R(0.8), cB = R(1.8) * I.alphaB - R(0.8);
    const R Qx = R(3) * (cR * dRx + cB * dBx), Qy = R(3) * (cR * dRy + cB * dBy);

    // moments of the shifted total populations
    R mT[Q9];
#pragma unroll
    for (int j = 0; j < Q9; j++) {
        R s = R(0);
#pragma unroll
        for (int i = 0; i < Q9; i++)
            if (m9(j, i) != 0) s += R(m9(j, i)) * fT[i];
        mT[j] = s;
    }
    // non-equilibrium part m - m^eq (rows e, epsilon in deviation form:
    // m = mT + moments of the shift; m^eq summed over the two colours)
    const R u2 = ux * ux + uy * uy;
    const R aBm = R(3.6) * I.alphaB + R(0.4), aRm = R(3.6) * I.alphaR + R(0.4);
    const R bBm = R(5.4) * I.alphaB - R(1.4), bRm = R(5.4) * I.alphaR - R(1.4);
    const R qco = R(-1.8) * (I.alphaR * rR + I.alphaB * rB) - R(0.2) * rho;
    R neq[Q9];
    neq[0] = R(0);
    // the shift of a flag-0 cell is the pure blue rest state, of a flag-1 cell
    // the pure red one, whose e and epsilon moments cancel the majority term
    if (fl == 0) {
        neq[1] = mT[1] + devmaj * aBm + rR * aRm - R(3) * rho * u2;
        neq[2] = mT[2] - devmaj * bBm - rR * bRm + R(3) * rho * u2;
    } else {
        neq[1] = mT[1] + devmaj * aRm + rB * aBm - R(3) * rho * u2;
        neq[2] = mT[2] - devmaj * bRm - rB * bBm + R(3) * rho * u2;
    }
    neq[1] += I.mcor1[fl];
    neq[2] += I.mcor2[fl];
    neq[3] = R(0);
    neq[4] = mT[4] - qco * ux;
    neq[5] = R(0);
    neq[6] = mT[6] - qco * uy;
    neq[7] = mT[7] - rho * (ux * ux - uy * uy);
    neq[8] = mT[8] - rho * ux * uy;

    // relaxation (Eq. 38) with s_v from the mixture viscosity (Eq. 43)
    const R rN = colour_fn(I, rR, rB);
    const R inv_mu = (R(1) + rN) * I.inv_2muR + (R(1) - rN) * I.inv_2muB;
    const R pk = rR * I.cs2R + rB * I.cs2B;
    const R sv = fdiv(R(1), R(0.5) + fdiv(R(1), inv_mu * pk));
    const R Sd[Q9] = {R(0), R(1.25), R(1.14), R(0), R(1.6), R(0), R(1.6), sv, sv};
    // forcing moments of Eq. 4 (closed form for D2Q9)
    const R uF = ux * Fx + uy * Fy;
    const R Fh[Q9] = {R(0), R(6) * uF, R(-6) * uF, Fx, -Fx, Fy, -Fy,
                      R(2) * (ux * Fx - uy * Fy), ux * Fy + uy * Fx};
    const R Cm[Q9] = {R(0), R(3) * (Qx + Qy), R(0), R(0), R(0), R(0), R(0), Qx - Qy, R(0)};
    R dm[Q9];
#pragma unroll
    for (int j = 0; j < Q9; j++)
        dm[j] = (-Sd[j] * neq[j] + (R(1) - R(0.5) * Sd[j]) * (Cm[j] + Fh[j])) *
                (R(1) / R(mnorm9(j)));

    // post-collision total minus shift
    R post[Q9];
    CSum<R> rdc;
#pragma unroll
    for (int i = 0; i < Q9; i++) {
        R s = fT[i];
#pragma unroll
        for (int j = 0; j < Q9; j++)
            if (m9(j, i) != 0) s += R(m9(j, i)) * dm[j];
        post[i] = s;
        rdc.add(shift_of(I, i, fl) + s);
    }
    const R rdag = rdc.value();
    // recolouring (Eqs. 11-12) of the minority colour; the majority is the
    // total minus it.  Segregation weight f_i^eq(rho, 0)/rho: for the
    // alpha-model its moving components are w_i * 3 p / rho with
    // p = sum_k rho^k (c_s^k)^2.  The split uses the post-collision total
    // rdag = sum_i f_i^dagger (= rho up to rounding) so that the colour mass
    // is conserved without a systematic rounding bias.
    const R ggx = I.gx[c], ggy = I.gy[c];
    const R seg = I.beta * rR * rB * R(3) * pk *
                  frsq(ggx * ggx + ggy * ggy + I.eps_n * I.eps_n) * fdiv(R(1), rho * rho);
    const R fr = fdiv(rmin, rdag);
    const R sg = fl ? R(-1) : R(1);
    // moving populations as stored; the rest populations close the cell's
    // total and minority mass on the pre-collision values (collision keeps
    // the total, recolouring each colour): every rounding residual of the
    // step stays in the cell
    CSum<R> sT, sM;
    const unsigned int rk = rest_key(c, rest_salt(0, I.ctl->step)), rs = pop_seed(rk);
#pragma unroll
    for (int i = 1; i < Q9; i++) {
        const R segi = seg * w9<R>(i) * (R(ex9(i)) * ggx + R(ey9(i)) * ggy);
        sT.add(stq_r<R, P>(I, I.gT, i, c, post[i], pop_r(rs, 2 * i)));
        sM.add(stq_r<R, P>(I, I.gM, i, c, fr * (I.shift[i] + post[i]) + sg * segi,
                           pop_r(rs, 2 * i + 1)));
    }
    I.gT0[c] = rest_close(mo.dr_s, mo.dr_c, sT.s, sT.c, R(0), rest_u(rk, 0));
    I.gM0[c] = rest_close(mo.rm_s, mo.rm_c, sM.s, sM.c, R(0), rest_u(rk, 1));
    I.gflag[c] = (uint8_t)fl;
}

// the explicit surfactant terms and the collision in one pass: both read
// only what k_force and the previous stream / grad kernels wrote, and they
// write disjoint fields
template <typename R, typename P>
__global__ void __launch_bounds__(256, 4) k_fdcollide2(Inst<R> I) {
    pdl_wait();
    pdl_trigger();
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (I.transport) fd2_cell(I, x, y, nullptr, nullptr);
    collide2_cell<R, P>(I, x, y);
}

template <typename R, typename P>
__global__ void k_collide2(Inst<R> I) {
    collide2_cell<R, P>(I, blockIdx.x * blockDim.x + threadIdx.x, blockIdx.y * blockDim.y + threadIdx.y);
}

// ---------------------------------------------------------------------------
// k_stream: f_i(x, t+1) = f_i^post(x - e_i) (Eq. 13, pull form); a link that
// crosses a wall is reflected (half-way bounce-back), a moving wall adds
// 2 w_i rho^k (e_i . u_w) / c_s^2.  Stores the moments at t+1.
// ---------------------------------------------------------------------------
template <typename R, typename P>
__device__ __forceinline__ void stream2_cell(const Inst<R> &I, int x, int y) {
    if (x >= I.nx || y >= I.ny) return;
    long long c = (long long)y * I.pitch + x;
    const int flc = I.gflag[c];
    const Ax X = make_ax(x, I.nx, I.wall[0], 1), Y = make_ax(y, I.ny, I.wall[1], 2);
    // 1. the streamed (total, minority) pairs as stored at their sources
    //    (i = 0 stays in its own cell); a link that crosses a wall reflects
    //    the cell's own opposite population; one crossing only mirror planes
    //    brings the mirrored population of the mirrored cell.  slow: bit i
    //    set where the source's flag differs from the cell's or the link
    //    crosses a moving wall.
    R t[Q9], m[Q9];
    unsigned slow = 0, fbits = 0;
    // (branch-free: a reflected link reads the cell's own opposite
    // population, so that every load of the loop can be in flight at once)
#pragma unroll
    for (int i = 0; i < Q9; i++) {
        int refl, sx, sy;
        const long long j = nbx2(I, X, Y, -ex9(i), -ey9(i), refl, sx, sy);
        if (i == 0) {
            t[0] = I.gT0[c];
            m[0] = I.gM0[c];
            continue;
        }
        const int bb = refl & I.bbmask;
        const long long src = bb ? c : j;
        const long long k = (long long)(bb ? opp9(i) : mir9(i, refl)) * I.plane + src;
        t[i] = ldp<R, P>(I, I.gT, k);
        m[i] = ldp<R, P>(I, I.gM, k);
        const int fj = I.gflag[src];
        fbits |= (unsigned)fj << i;
        // (a static wall returns the cell's own opposite population unchanged:
        // the fast path's plain move; a moving wall adds its momentum term)
        if (fj != flc || (bb & I.mvmask)) slow |= 1u << i;
    }
    fbits |= (unsigned)flc;  // (i = 0: the cell's own flag)
    // 2. fast path: every population moves unchanged (no rounding anywhere);
    //    the cell keeps its flag unless its minority has become the majority
    if (!slow) {
        CSum<R> tot, mn;
        R jx = R(0), jy = R(0);
#pragma unroll
        for (int i = 0; i < Q9; i++) {
            tot.add(t[i]);
            mn.add(m[i]);
            if (ex9(i)) jx += R(ex9(i)) * t[i];
            if (ey9(i)) jy += R(ey9(i)) * t[i];
        }
        const R rmin = mn.value(), rmaj = (I.rho_s[flc] - rmin) + tot.value();
        const R rR = flc ? rmaj : rmin, rB = flc ? rmin : rmaj;
        if (minority(I, rR, rB) == flc) {
#pragma unroll
            for (int i = 1; i < Q9; i++) {
                stp<R, P>(I, I.fT, (long long)i * I.plane + c, t[i]);
                stp<R, P>(I, I.fM, (long long)i * I.plane + c, m[i]);
            }
            I.fT0[c] = t[0];
            I.fM0[c] = m[0];
            I.flag[c] = (uint8_t)flc;
            I.rhoR[c] = rR;
            I.rhoB[c] = rB;
            I.rhoN[c] = colour_fn(I, rR, rB);
            I.jx[c] = jx;
            I.jy[c] = jy;
            return;
        }
    }
    // 3. general path: colours re-split where the flags differ, moving-wall
    //    terms (2 w_i rho^k (e_i . u_w) / c_s^2) added; every value carried
    //    as hi + lo (TwoSum errors), and the rest populations close the
    //    cell's total and minority mass exactly
    const R rRc = I.rhoR[c], rBc = I.rhoB[c];
    R fR[Q9], fB[Q9];
    R loT = R(0), loR = R(0), loB = R(0);
#pragma unroll
    for (int i = 0; i < Q9; i++) {
        const int fj = (fbits >> i) & 1;
        R tlo = R(0), mlo = R(0);
        R sh = shift_of(I, i, fj);
        if ((slow >> i) & 1) {
            int refl, sx, sy;
            nbx2(I, X, Y, -ex9(i), -ey9(i), refl, sx, sy);
            refl &= I.bbmask;  // (mirror planes reflect without a wall term)
            if (refl) {
                R uwx = R(0), uwy = R(0);
                int nw = 0;
                if (refl & 1) {
                    const R *w = sx < 0 ? I.uw_lo[0] : I.uw_hi[0];
                    uwx += w[0];
                    uwy += w[1];
                    nw++;
                }
                if (refl & 2) {
                    const R *w = sy < 0 ? I.uw_lo[1] : I.uw_hi[1];
                    uwx += w[0];
                    uwy += w[1];
                    nw++;
                }
                const R eu = (R(ex9(i)) * uwx + R(ey9(i)) * uwy) / R(nw);
                const R mw = R(2) * w9<R>(i) * eu * R(3);
                t[i] = two_sum(t[i], mw * (rRc + rBc), tlo);
                m[i] = two_sum(m[i], mw * (flc ? rBc : rRc), mlo);
                sh = I.shift[i];
            }
        }
        loT += tlo;
        R e1, e2;
        const R o = two_sum(two_sum(sh, t[i], e1), -m[i], e2);
        const R olo = (e1 + e2) + (tlo - mlo);
        fR[i] = fj ? o : m[i];
        fB[i] = fj ? m[i] : o;
        loR += fj ? olo : mlo;
        loB += fj ? mlo : olo;
    }
    R rR = R(0), rB = R(0);
#pragma unroll
    for (int i = 0; i < Q9; i++) {
        rR += fR[i];
        rB += fB[i];
    }
    const int fl = minority(I, rR, rB);
    // a change of flag re-expresses the rest population against the new
    // rest shift (the moving shifts are common to both flags)
    if (fl != flc) {
        R d1, d2;
        const R d = two_sum(I.shift0[flc], -I.shift0[fl], d1);
        t[0] = two_sum(d, t[0], d2);
        loT += d1 + d2;
    }
    // stored: the high parts; their rounding and every low part go to the
    // rest populations through the remainder
    R fT[Q9], fM[Q9];
    CSum<R> gT, gM, sT, sM;
    const R loM = fl ? loB : loR;
    const unsigned int rk = rest_key(c, rest_salt(1, I.ctl->step)), rs = pop_seed(rk);
#pragma unroll
    for (int i = 0; i < Q9; i++) {
        const R mh = fl ? fB[i] : fR[i];
        gT.add(t[i]);
        gM.add(mh);
        if (i) {
            fT[i] = stq_r<R, P>(I, I.fT, i, c, t[i], pop_r(rs, 2 * i));
            fM[i] = stq_r<R, P>(I, I.fM, i, c, mh, pop_r(rs, 2 * i + 1));
            sT.add(fT[i]);
            sM.add(fM[i]);
        }
    }
    fT[0] = rest_close(gT.s, gT.c, sT.s, sT.c, loT, rest_u(rk, 0));
    fM[0] = rest_close(gM.s, gM.c, sM.s, sM.c, loM, rest_u(rk, 1));
    I.fT0[c] = fT[0];
    I.fM0[c] = fM[0];
    I.flag[c] = (uint8_t)fl;
    store_moments(I, c, fT, fM, fl);
}

template <typename R, typename P>
__global__ void k_stream2(Inst<R> I) {
    pdl_wait();
    pdl_trigger();
    stream2_cell<R, P>(I, blockIdx.x * blockDim.x + threadIdx.x, blockIdx.y * blockDim.y + threadIdx.y);
}

// ---------------------------------------------------------------------------
// SOR (Sec. 2.2: relaxation factor 1.2) for (w - h L_w) x = rhs on psi
// (w = a + eps_w, h = Ds/2) and C (w = chi + eps_w, h = Db/2).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void atomic_max_pos(unsigned long long *p, double v) {
    atomicMax(p, (unsigned long long)__double_as_longlong(v));
}

template <typename R>
__device__ __forceinline__ bool sweep_converged(const Ctl *ctl, int k, double tol) {
    double dp = __longlong_as_double((long long)ctl->sweep[k][0]);
    double dc = __longlong_as_double((long long)ctl->sweep[k][1]);
    double xp = __longlong_as_double((long long)ctl->sweep[k][2]);
    double xc = __longlong_as_double((long long)ctl->sweep[k][3]);
    return dp <= tol * xp && dc <= tol * xc;
}

// ---------------------------------------------------------------------------
// k_sor_tb2: K red-black SOR sweeps per launch with temporal blocking.  A block
// loads its TX x TY tile plus a halo of H = 2K cells into shared memory and
// sweeps there; a red or black half-sweep spreads the error of the stale
// region border by one cell, so after K sweeps the tile interior holds exactly
// the values global red-black SOR would have.  psi and C are read from one
// global buffer and the interior is written to the other (rounds alternate),
// so no block reads values written by the same round.  Round r skips when
// round r-1 met the tolerance on its last sweep.
//
// Two forms of the tile (same iterates):
//  - checkerboard (every periodic axis of even length, the usual case): the
//    colour of region cell (rx, ry) is (rx + ry) & 1, since tile origins are
//    even, and no two cells of one colour are neighbours, so a half-sweep
//    updates its colour in place.  Shared arrays are split by colour,
//    A[c][ry][rx / 2], so the cells a warp updates and the neighbours it
//    reads are consecutive words; half-sweep t of 2K updates only the
//    rectangle of margin 2K - 1 - t around the tile, the cells that still
//    reach the tile interior;
//  - list (an odd periodic axis): cells of one colour meet across the seam,
//    so the updates of a half-sweep are staged in registers and written after
//    a barrier (a deterministic Jacobi step within the colour), over lists of
//    the cells of each colour.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool last_block(unsigned int *ticket, unsigned int nblocks);

template <typename R, int TX, int TY, int K, int BS>
struct SorTile {
    static constexpr int H = 2 * K, RX = TX + 2 * H, RY = TY + 2 * H, NR = RX * RY;
    // checkerboard form: a colour plane of RY rows of RXH words, planes NHP
    // apart (16 words of padding put the planes' banks half a warp apart)
    static constexpr int RXH = RX / 2, NH = RY * RXH, NHP = NH + 16;
    static_assert(TX % 2 == 0 && TY % 2 == 0, "SOR tiles have even sides");
    // per region cell: psi, C, rhs psi, rhs C, inverse diagonals (2), face
    // coefficients to the +x and +y neighbours (2 fields x 2), one flag byte;
    // the list form adds the cell lists of the two colours (2-byte indices)
    static constexpr size_t list_bytes() { return (size_t)NR * (10 * sizeof(R) + 1 + 2 * 2) + 16; }
    static constexpr size_t cb_bytes() { return (size_t)2 * NHP * (10 * sizeof(R) + 1) + 16; }
    static constexpr size_t smem_bytes() {
        return list_bytes() > cb_bytes() ? list_bytes() : cb_bytes();
    }
};

// the blocked SOR variants: tile TX x TY, K sweeps a launch, BS threads.
// A larger K halves the launches at the price of a wider halo (2K); more
// threads a block put more loads of the region in flight.
//   v:   0      1     2      3      4      5      6      7      8
//   TX:  32     64    16     32     32     32     64     32     32
//   TY:  16     8     16     16     32     32     16     32     16
//   K:   2      2     2      4      4      4      4      6      8
//   BS:  256    256   256    256    256    512    512    512    512
// (variants 7 and 8 exceed the shared memory of a block in double precision)
constexpr int kSorVariants = 9;
__host__ __device__ constexpr int sor_vtx(int v) { return (v == 1 || v == 6) ? 64 : (v == 2 ? 16 : 32); }
__host__ __device__ constexpr int sor_vty(int v) {
    return v == 1 ? 8 : ((v == 4 || v == 5 || v == 7) ? 32 : 16);
}
__host__ __device__ constexpr int sor_vk(int v) { return v == 8 ? 8 : (v == 7 ? 6 : (v >= 3 ? 4 : 2)); }
__host__ __device__ constexpr int sor_vbs(int v) { return v >= 5 ? 512 : 256; }

// convergence of a round: the largest update of its last sweep is within
// sor_tol of the largest value, or (single precision) the updates stopped
// shrinking at a level within 8 sor_tol, i.e. at the rounding floor
template <typename R>
__device__ __forceinline__ bool round_converged(const Ctl *ctl, int r, double tol) {
    if (sweep_converged<R>(ctl, r, tol)) return true;
    if (sizeof(R) != 4 || r == 0) return false;
    if (!sweep_converged<R>(ctl, r, 8 * tol)) return false;
    double d0 = fmax(__longlong_as_double((long long)ctl->sweep[r - 1][0]),
                     __longlong_as_double((long long)ctl->sweep[r - 1][1]));
    double d1 = fmax(__longlong_as_double((long long)ctl->sweep[r][0]),
                     __longlong_as_double((long long)ctl->sweep[r][1]));
    return d1 >= 0.5 * d0;
}

// block maxima of the last sweep (|dpsi|, |dC|, |psi|, |C|) -> round slot
template <typename R, int BS>
__device__ __forceinline__ void sor_fold_maxima(const Inst<R> &I, int round, R v[4]) {
    __shared__ R sh[4][BS / 32];
    const int tid = threadIdx.x;
#pragma unroll
    for (int q = 0; q < 4; q++)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[q] = fmax(v[q], __shfl_down_sync(0xffffffffu, v[q], o));
    if ((tid & 31) == 0)
        for (int q = 0; q < 4; q++) sh[q][tid >> 5] = v[q];
    __syncthreads();
    if (tid == 0)
        for (int q = 0; q < 4; q++) {
            R m = R(0);
            for (int w = 0; w < BS / 32; w++) m = fmax(m, sh[q][w]);
            atomic_max_pos(&I.ctl->sweep[round][q], double(m));
        }
}

// checkerboard form of a tile (see above).  The two systems are swept
// together, so each region slot keeps its psi and C values side by side
// (one 2-vector load a neighbour): X = (psi, C), Bv = right-hand sides,
// Iv = inverse diagonals, FX / FY = face coefficients towards +x / +y.
template <typename R, int TX, int TY, int K, int BS>
__device__ __forceinline__ void sor_tile2_cb(const Inst<R> &I, int round, int bx, int by,
                                             unsigned char *smem_raw, R *tot, bool keep) {
    using T = SorTile<R, TX, TY, K, BS>;
    using V = typename Vec2<R>::T;
    constexpr int RX = T::RX, RY = T::RY, H = T::H, RXH = T::RXH, NH = T::NH, NHP = T::NHP;
    constexpr int NS = 2 * NHP;
    V *X = (V *)smem_raw, *Bv = X + NS, *Iv = Bv + NS, *FX = Iv + NS, *FY = FX + NS;
    uint8_t *fl = (uint8_t *)(FY + NS);                // 1: in the domain
    const int tid = threadIdx.x;
    const int x0 = bx * TX - H, y0 = by * TY - H;      // even
    const bool odd = ((round + I.sor_phase) & 1) != 0;
    const R *pin = odd ? I.psi2 : I.psi;
    const R *cin = odd ? I.C2 : I.C;
    R *pout = odd ? I.psi : I.psi2;
    R *cout = odd ? I.C : I.C2;
    const V zero = {R(0), R(0)};
    // The coefficients (faces, inverse diagonals) depend only on a and chi,
    // fixed during the solve: round 0 builds them from a and chi (steps 1-3)
    // and stores those of its tile interior; later rounds load them (step 1').
    const bool first = round == 0 || I.sfx == nullptr;
    if (!first && keep) {
        // 1''. the block took this same tile in the round before: the
        //      right-hand sides and coefficients are still in shared memory,
        //      and so are psi, C of the cells it owns (the values it wrote
        //      back); only the other region slots are reloaded
        for (int q = tid; q < RX * RY; q += BS) {
            const int rx = q % RX, ry = q / RX;
            if (rx >= H && rx < H + TX && ry >= H && ry < H + TY && x0 + rx < I.nx &&
                y0 + ry < I.ny)
                continue;
            int refl = 0, sx, sy;
            const int Xc = map_axis(x0 + rx, I.nx, I.wall[0], 1, refl, sx);
            const int Yc = map_axis(y0 + ry, I.ny, I.wall[1], 2, refl, sy);
            const int s = ((rx + ry) & 1) * NHP + ry * RXH + (rx >> 1);
            if (!refl) {
                const long long c = (long long)Yc * I.pitch + Xc;
                X[s] = V{__ldcg(&pin[c]), __ldcg(&cin[c])};
            } else {
                X[s] = zero;
            }
        }
        __syncthreads();
    } else if (!first) {
        // 1'. load psi, C, the right-hand sides and the coefficients, in row
        //     order; zero outside the domain.  psi and C change between the
        //     rounds of one launch: they are read through L2, never from a
        //     line an earlier round left in L1.
        for (int q = tid; q < RX * RY; q += BS) {
            const int rx = q % RX, ry = q / RX;
            int refl = 0, sx, sy;
            const int Xc = map_axis(x0 + rx, I.nx, I.wall[0], 1, refl, sx);
            const int Yc = map_axis(y0 + ry, I.ny, I.wall[1], 2, refl, sy);
            const int s = ((rx + ry) & 1) * NHP + ry * RXH + (rx >> 1);
            if (!refl) {
                const long long c = (long long)Yc * I.pitch + Xc;
                X[s] = V{__ldcg(&pin[c]), __ldcg(&cin[c])};
                Bv[s] = V{I.rpsi[c], I.rC[c]};
                FX[s] = V{I.sfx[c], I.scx[c]};
                FY[s] = V{I.sfy[c], I.scy[c]};
                Iv[s] = V{I.sip[c], I.sic[c]};
            } else {
                X[s] = Bv[s] = FX[s] = FY[s] = Iv[s] = zero;
            }
        }
        __syncthreads();
    } else {
        // 1. load in row order (coalesced); Iv holds the weights a + eps,
        //    chi + eps for now, zero outside the domain.  A thread loads U cells
        //    into registers before it stores any, so that their loads are in
        //    flight together (a store to shared memory would otherwise order the
        //    next cell's loads behind it).
        constexpr int U = 3;
        for (int q0 = tid; q0 < RX * RY; q0 += U * BS) {
            R vv[U][6];
            int ss[U];
            bool in[U];
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int q = q0 + u * BS;
                in[u] = false;
                ss[u] = -1;
                if (q >= RX * RY) continue;
                const int rx = q % RX, ry = q / RX;
                int refl = 0, sx, sy;
                const int Xc = map_axis(x0 + rx, I.nx, I.wall[0], 1, refl, sx);
                const int Yc = map_axis(y0 + ry, I.ny, I.wall[1], 2, refl, sy);
                ss[u] = ((rx + ry) & 1) * NHP + ry * RXH + (rx >> 1);
                in[u] = !refl;
                if (!refl) {
                    const long long c = (long long)Yc * I.pitch + Xc;
                    vv[u][0] = __ldcg(&pin[c]);
                    vv[u][1] = __ldcg(&cin[c]);
                    vv[u][2] = I.rpsi[c];
                    vv[u][3] = I.rC[c];
                    vv[u][4] = __ldcg(&I.a[c]);
                    vv[u][5] = __ldcg(&I.chi[c]);
                }
            }
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int s = ss[u];
                if (s < 0) continue;
                if (in[u]) {
                    X[s] = V{vv[u][0], vv[u][1]};
                    Bv[s] = V{vv[u][2], vv[u][3]};
                    Iv[s] = V{vv[u][4] + I.eps_w, vv[u][5] + I.eps_w};
                } else {
                    X[s] = Bv[s] = Iv[s] = zero;
                }
                fl[s] = in[u];
            }
        }
        __syncthreads();
        // 2. face coefficients h (w_c + w_nb)/2 of Eq. 28 towards +x and +y; zero
        //    across a wall or the region edge
        const R hp = R(0.5) * I.Ds, hc = R(0.5) * I.Db;
        for (int q = tid; q < 2 * NH; q += BS) {
            const int c = q >= NH, r = q - c * NH, ry = r / RXH, j = r - ry * RXH;
            const int rx = 2 * j + ((c ^ ry) & 1);
            const int s = c * NHP + r, o = (1 - c) * NHP + ry * RXH;
            const bool in = fl[s];
            const bool ex = in && rx < RX - 1 && fl[o + ((rx + 1) >> 1)];
            const bool ny = in && ry < RY - 1 && fl[o + RXH + j];
            const int e = o + ((rx + 1) >> 1), n = o + RXH + j;
            const V ws = Iv[s], we = Iv[e], wn = Iv[n];
            FX[s] = ex ? V{hp * R(0.5) * (ws.x + we.x), hc * R(0.5) * (ws.y + we.y)} : zero;
            FY[s] = ny ? V{hp * R(0.5) * (ws.x + wn.x), hc * R(0.5) * (ws.y + wn.y)} : zero;
        }
        __syncthreads();
        // 3. inverse diagonals w + sum of the four faces (zero outside the domain,
        //    where the weights are zero: those cells stay zero in every sweep)
        for (int q = tid; q < 2 * NH; q += BS) {
            const int c = q >= NH, r = q - c * NH, ry = r / RXH, j = r - ry * RXH;
            const int rx = 2 * j + ((c ^ ry) & 1);
            const int s = c * NHP + r, o = (1 - c) * NHP + ry * RXH;
            if (!fl[s]) continue;
            const int w = o + ((rx - 1) >> 1), so = o - RXH + j;
            const V fx = FX[s], fy = FY[s];
            const V fxw = rx > 0 ? FX[w] : zero, fyso = ry > 0 ? FY[so] : zero;
            const R sp_ = fx.x + fy.x + fxw.x + fyso.x;
            const R sc_ = fx.y + fy.y + fxw.y + fyso.y;
            const V ws = Iv[s];
            Iv[s] = V{fdiv(R(1), ws.x + sp_), fdiv(R(1), ws.y + sc_)};
        }
        __syncthreads();
    }
    // 2K half-sweeps in place; half-sweep t updates colour t & 1 over the
    // rectangle of margin m = 2K - 1 - t around the tile
    R v[4] = {R(0), R(0), R(0), R(0)};  // maxima of the last sweep (never FP64 per cell)
#pragma unroll
    for (int t = 0; t < 2 * K; t++) {
        const int c = t & 1, m = 2 * K - 1 - t;
        const int lo = H - m, xhi = H + TX + m, yhi = H + TY + m;  // lo >= 1
        const int jlo = lo >> 1, jn = ((xhi - 1) >> 1) - jlo + 1;
        const int n = (yhi - lo) * jn;
        const bool last = t >= 2 * K - 2;
        for (int idx = tid; idx < n; idx += BS) {
            const int ry = lo + idx / jn, j = jlo + idx % jn;
            const int rx = 2 * j + ((c ^ ry) & 1);
            if (rx < lo || rx >= xhi) continue;
            const int s = c * NHP + ry * RXH + j, o = (1 - c) * NHP + ry * RXH;
            const int e = o + ((rx + 1) >> 1), w = o + ((rx - 1) >> 1);
            const int nn = o + RXH + j, so = o - RXH + j;
            const V xe = X[e], xn = X[nn], xw = X[w], xso = X[so];
            const V fx = FX[s], fy = FY[s], fxw = FX[w], fyso = FY[so];
            const V b = Bv[s], iv = Iv[s], x0v = X[s];
            const R op = b.x + fx.x * xe.x + fy.x * xn.x + fxw.x * xw.x + fyso.x * xso.x;
            const R oc = b.y + fx.y * xe.y + fy.y * xn.y + fxw.y * xw.y + fyso.y * xso.y;
            const R dp = I.omega * (op * iv.x - x0v.x);
            const R dc = I.omega * (oc * iv.y - x0v.y);
            const R p1 = x0v.x + dp, c1 = x0v.y + dc;
            X[s] = V{p1, c1};
            if (last && rx >= H && rx < H + TX && ry >= H && ry < H + TY && x0 + rx < I.nx &&
                y0 + ry < I.ny) {
                v[0] = fmax(v[0], fabs(dp));
                v[1] = fmax(v[1], fabs(dc));
                v[2] = fmax(v[2], fabs(p1));
                v[3] = fmax(v[3], fabs(c1));
            }
        }
        __syncthreads();
    }
    // tile interior back to the other buffer, in row order
    for (int q = tid; q < TX * TY; q += BS) {
        const int rx = H + q % TX, ry = H + q / TX;
        const int gx = x0 + rx, gy = y0 + ry;
        if (gx >= I.nx || gy >= I.ny) continue;
        const int s = ((rx + ry) & 1) * NHP + ry * RXH + (rx >> 1);
        const long long c = (long long)gy * I.pitch + gx;
        const V xs = X[s];
        pout[c] = xs.x;
        cout[c] = xs.y;
        if (tot) {
            comp_add_prod(tot[0], tot[1], __ldcg(&I.a[c]) + I.eps_w, xs.x);
            comp_add_prod(tot[0], tot[1], __ldcg(&I.chi[c]) + I.eps_w, xs.y);
        }
        if (first && I.sfx && !keep) {
            const V fx = FX[s], fy = FY[s], iv = Iv[s];
            I.sfx[c] = fx.x;
            I.scx[c] = fx.y;
            I.sfy[c] = fy.x;
            I.scy[c] = fy.y;
            I.sip[c] = iv.x;
            I.sic[c] = iv.y;
        }
    }
    sor_fold_maxima<R, BS>(I, round, v);
}

// list form of a tile (see above)
template <typename R, int TX, int TY, int K, int BS>
__device__ __forceinline__ void sor_tile2_list(const Inst<R> &I, int round, int bx, int by,
                                               unsigned char *smem_raw, R *tot) {
    using T = SorTile<R, TX, TY, K, BS>;
    constexpr int RX = T::RX, RY = T::RY, NR = T::NR, H = T::H;
    R *sp = (R *)smem_raw, *sc = sp + NR, *bp = sc + NR, *bc = bp + NR;
    R *ip = bc + NR, *ic = ip + NR;                    // 1 / diagonal
    R *fpx = ic + NR, *fpy = fpx + NR, *fcx = fpy + NR, *fcy = fcx + NR;  // faces +x, +y
    uint8_t *fl = (uint8_t *)(fcy + NR);
    uint16_t *list = (uint16_t *)(((uintptr_t)(fl + NR) + 1) & ~(uintptr_t)1);
    __shared__ int count[2];
    const int tid = threadIdx.x;
    const int x0 = bx * TX - H, y0 = by * TY - H;
    const bool odd = ((round + I.sor_phase) & 1) != 0;
    const R *pin = odd ? I.psi2 : I.psi;
    const R *cin = odd ? I.C2 : I.C;
    R *pout = odd ? I.psi : I.psi2;
    R *cout = odd ? I.C : I.C2;
    if (tid < 2) count[tid] = 0;
    // 1. load.  flags: bit0 in the domain, bit1 colour, bit6 tile interior
    //    owned here; ip / ic hold the weights a + eps, chi + eps for now
    for (int q = tid; q < NR; q += BS) {
        int rx = q % RX, ry = q / RX;
        int gx = x0 + rx, gy = y0 + ry;
        int refl = 0, sx, sy;
        int X = map_axis(gx, I.nx, I.wall[0], 1, refl, sx);
        int Y = map_axis(gy, I.ny, I.wall[1], 2, refl, sy);
        uint8_t f = 0;
        if (!refl) {
            long long c = (long long)Y * I.pitch + X;
            f = 1 | (((X + Y) & 1) << 1);
            sp[q] = __ldcg(&pin[c]);
            sc[q] = __ldcg(&cin[c]);
            bp[q] = I.rpsi[c];
            bc[q] = I.rC[c];
            ip[q] = I.a[c] + I.eps_w;
            ic[q] = I.chi[c] + I.eps_w;
            if (rx >= H && rx < H + TX && ry >= H && ry < H + TY && gx >= 0 && gx < I.nx &&
                gy >= 0 && gy < I.ny)
                f |= 64;
        } else {
            sp[q] = sc[q] = bp[q] = bc[q] = ip[q] = ic[q] = R(0);
        }
        fl[q] = f;
    }
    __syncthreads();
    // 2. face coefficients h (w_c + w_nb)/2 of Eq. 28 towards +x and +y; zero
    //    across a wall or the region edge (no flux, no branch in the sweeps)
    const R hp = R(0.5) * I.Ds, hc = R(0.5) * I.Db;
    for (int q = tid; q < NR; q += BS) {
        int rx = q % RX, ry = q / RX;
        const bool in = fl[q] & 1;
        const bool ex = in && rx < RX - 1 && (fl[q + 1] & 1);
        const bool ny = in && ry < RY - 1 && (fl[q + RX] & 1);
        fpx[q] = ex ? hp * R(0.5) * (ip[q] + ip[q + 1]) : R(0);
        fcx[q] = ex ? hc * R(0.5) * (ic[q] + ic[q + 1]) : R(0);
        fpy[q] = ny ? hp * R(0.5) * (ip[q] + ip[q + RX]) : R(0);
        fcy[q] = ny ? hc * R(0.5) * (ic[q] + ic[q + RX]) : R(0);
    }
    __syncthreads();
    // 3. inverse diagonals w + sum of the four faces, and the lists of the
    //    cells of each colour that can be updated (not on the region border)
    for (int q = tid; q < NR; q += BS) {
        int rx = q % RX, ry = q / RX;
        uint8_t f = fl[q];
        if (!(f & 1)) continue;
        R sp_ = fpx[q] + fpy[q] + (rx > 0 ? fpx[q - 1] : R(0)) + (ry > 0 ? fpy[q - RX] : R(0));
        R sc_ = fcx[q] + fcy[q] + (rx > 0 ? fcx[q - 1] : R(0)) + (ry > 0 ? fcy[q - RX] : R(0));
        ip[q] = fdiv(R(1), ip[q] + sp_);
        ic[q] = fdiv(R(1), ic[q] + sc_);
        if (rx > 0 && rx < RX - 1 && ry > 0 && ry < RY - 1) {
            int col = (f >> 1) & 1;
            int slot = atomicAdd(&count[col], 1);
            list[col * NR + slot] = (uint16_t)q;
        }
    }
    __syncthreads();
    // K red-black sweeps; a half-sweep stages its updates in registers
    R v[4] = {R(0), R(0), R(0), R(0)};  // maxima of the last sweep (never FP64 per cell)
    constexpr int PER = (NR / 2 + BS) / BS + 1;
    for (int s = 0; s < K; s++) {
        for (int colour = 0; colour < 2; colour++) {
            const int n = count[colour];
            const uint16_t *L = list + colour * NR;
            R np[PER], nc[PER];
#pragma unroll
            for (int k = 0; k < PER; k++) {
                int idx = tid + k * BS;
                np[k] = R(0);
                nc[k] = R(0);
                if (idx >= n) continue;
                int q = L[idx];
                R op = bp[q] + fpx[q] * sp[q + 1] + fpy[q] * sp[q + RX] + fpx[q - 1] * sp[q - 1] +
                       fpy[q - RX] * sp[q - RX];
                R oc = bc[q] + fcx[q] * sc[q + 1] + fcy[q] * sc[q + RX] + fcx[q - 1] * sc[q - 1] +
                       fcy[q - RX] * sc[q - RX];
                R p0 = sp[q], c0 = sc[q];
                R dp = I.omega * (op * ip[q] - p0);
                R dc = I.omega * (oc * ic[q] - c0);
                np[k] = p0 + dp;
                nc[k] = c0 + dc;
                if (s == K - 1 && (fl[q] & 64)) {
                    v[0] = fmax(v[0], fabs(dp));
                    v[1] = fmax(v[1], fabs(dc));
                    v[2] = fmax(v[2], fabs(np[k]));
                    v[3] = fmax(v[3], fabs(nc[k]));
                }
            }
            __syncthreads();
#pragma unroll
            for (int k = 0; k < PER; k++) {
                int idx = tid + k * BS;
                if (idx >= n) continue;
                int q = L[idx];
                sp[q] = np[k];
                sc[q] = nc[k];
            }
            __syncthreads();
        }
    }
    // interior cells back to the other buffer
    for (int q = tid; q < NR; q += BS) {
        if (!(fl[q] & 64)) continue;
        int rx = q % RX, ry = q / RX;
        long long c = (long long)(y0 + ry) * I.pitch + (x0 + rx);
        pout[c] = sp[q];
        cout[c] = sc[q];
        if (tot) {
            comp_add_prod(tot[0], tot[1], __ldcg(&I.a[c]) + I.eps_w, sp[q]);
            comp_add_prod(tot[0], tot[1], __ldcg(&I.chi[c]) + I.eps_w, sc[q]);
        }
    }
    sor_fold_maxima<R, BS>(I, round, v);
}

// L2 prefetch of the lines tile (bx, by) of round `round` will load (the
// region of the tile and its halo, rows and columns inside the grid): a
// block that takes several tiles a round issues it for its next tile before
// it works on the current one, so that the next tile's loads find L2 rather
// than wait on DRAM one dependent round at a time.  The round's inputs are
// not written during the round, so the lines stay valid.
template <typename R, int TX, int TY, int K, int BS>
__device__ __forceinline__ void sor_prefetch_tile(const Inst<R> &I, int round, int bx, int by) {
    constexpr int H = SorTile<R, TX, TY, K, BS>::H;
    const bool odd = ((round + I.sor_phase) & 1) != 0;
    const int np = (round > 0 && I.sfx != nullptr) ? 10 : 6;
    const int xlo = max(bx * TX - H, 0), xhi = min(bx * TX + TX + H, I.nx);
    const int ylo = max(by * TY - H, 0), yhi = min(by * TY + TY + H, I.ny);
    if (xhi <= xlo || yhi <= ylo) return;
    const int lo = xlo * (int)sizeof(R), hi = xhi * (int)sizeof(R) - 1;  // bytes of a row
    const int nl = (hi - lo) / 128 + 2;                                  // lines a row (one spare)
    const int per = (yhi - ylo) * nl;
    for (int it = threadIdx.x; it < np * per; it += BS) {
        const int k = it / per, r0 = it - k * per, r = r0 / nl, l = r0 - r * nl;
        const R *b;
        switch (k) {
        case 0: b = odd ? I.psi2 : I.psi; break;
        case 1: b = odd ? I.C2 : I.C; break;
        case 2: b = I.rpsi; break;
        case 3: b = I.rC; break;
        case 4: b = np == 10 ? I.sfx : I.a; break;
        case 5: b = np == 10 ? I.scx : I.chi; break;
        case 6: b = I.sfy; break;
        case 7: b = I.scy; break;
        case 8: b = I.sip; break;
        default: b = I.sic; break;
        }
        const char *a = (const char *)(b + (size_t)(ylo + r) * I.pitch) + min(lo + 128 * l, hi);
        asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
    }
}

// one tile (bx, by) of round `round` of instance I, in smem_raw
// (SorTile::smem_bytes()); folds the tile's maxima into the round's slot.
// With tot (a thread's compensated sum hi, lo), the thread also adds the
// surfactant (a + eps) psi + (chi + eps) C of the tile cells it stores, each
// product exact as hi + lo.
// keep: the calling block takes this same tile in every round of the launch,
// so the checkerboard form keeps the tile's coefficients and right-hand sides
// in shared memory from round to round (identical iterates).
template <typename R, int TX, int TY, int K, int BS>
__device__ __forceinline__ void sor_tile2(const Inst<R> &I, int round, int bx, int by,
                                          unsigned char *smem_raw, R *tot = nullptr,
                                          bool keep = false) {
    if ((I.wall[0] || !(I.nx & 1)) && (I.wall[1] || !(I.ny & 1)))
        sor_tile2_cb<R, TX, TY, K, BS>(I, round, bx, by, smem_raw, tot, keep);
    else
        sor_tile2_list<R, TX, TY, K, BS>(I, round, bx, by, smem_raw, tot);
}

// ---------------------------------------------------------------------------
// Grid barrier of the one-launch SOR (k_sorfuse2, lbs_fused2.cuh): every
// block of a cooperative launch arrives, the last one releases the others.
// A barrier waits at most max_polls polls (the default, kBarrierPolls, is
// about a second), then reports ST_TIMEOUT and returns false.
// ---------------------------------------------------------------------------
constexpr long long kBarrierPolls = 1LL << 24;

// Grid barrier of a cooperative launch: every block adds one arrival to a
// counter that the kernel before the launch cleared, and waits until the
// count reaches nblocks times the barriers passed so far (target, kept by
// the caller): no block resets or flips anything, so the last arrival is
// seen after one write.  True in every thread of the block once every block
// arrived; false when the wait gave up (ST_TIMEOUT: the count then stays
// short of every later target, so the launch's later barriers give up too,
// and the next launch starts from a cleared counter).
__device__ __forceinline__ bool grid_barrier(Ctl *ctl, unsigned int nblocks,
                                             unsigned int &target, long long max_polls) {
    __shared__ int ok;
    target += nblocks;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        __threadfence();
        atomicAdd(&ctl->bar_count, 1u);
        const volatile unsigned int *count = &ctl->bar_count;
        long long polls = 0;
        while (*count < target) {
            if (++polls > max_polls) {
                ok = 0;
                atomicOr(&ctl->status, int(ST_TIMEOUT));
                break;
            }
            __nanosleep(32);
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

// decision after a round of instance ctl: converged, or out of rounds
template <typename R>
__device__ __forceinline__ bool sor_round_stop(Ctl *ctl, int round, double tol, int max_rounds) {
    const bool conv = round_converged<R>(ctl, round, tol);
    const bool stop = conv || round + 1 >= max_rounds;
    if (stop && !conv) ctl->status |= ST_NOCONV;
    return stop;
}

// loop: the WHILE node's handle in graph mode; eager_round >= 0 instead runs
// round eager_round of a host-side loop (returns at once once converged)
template <typename R, int TX, int TY, int K, int BS>
__global__ void __launch_bounds__(BS)
    k_sor_tb2(Inst<R> I, cudaGraphConditionalHandle loop, int max_rounds, int eager_round) {
    if (eager_round > 0 && I.ctl->sor_exec < eager_round) return;  // loop already ended
    const int round = I.ctl->sor_exec;  // rounds run so far in this solve
    extern __shared__ __align__(16) unsigned char smem_raw[];
    sor_tile2<R, TX, TY, K, BS>(I, round, blockIdx.x, blockIdx.y, smem_raw);
    const int tid = threadIdx.x;
    // the last block to finish decides whether the loop runs another round
    const unsigned int nb = gridDim.x * gridDim.y;
    if (!last_block(&I.ctl->sor_ticket, nb)) return;
    if (tid != 0) return;
    Ctl *ctl = I.ctl;
    ctl->sor_ticket = 0;
    const bool stop = sor_round_stop<R>(ctl, round, double(I.sor_tol), max_rounds);
    if (eager_round < 0) {
        ctl->sor_exec = round + 1;
        if (stop) cudaGraphSetConditional(loop, 0);
    } else {
        // eager: sor_exec counts finished rounds; a stop freezes it one below
        // the next launch's index so that the later launches return at once
        ctl->sor_exec = stop ? -(round + 1) - 1000000 : round + 1;
    }
}

// ---------------------------------------------------------------------------
// Deterministic FP64 reductions: per-block partials, the last block to arrive
// sums them in block order.
// ---------------------------------------------------------------------------
template <int BS, int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double *out /* K, thread 0 */) {
    __shared__ double sh[K][BS / 32];
#pragma unroll
    for (int q = 0; q < K; q++) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
    }
    int t = threadIdx.x + threadIdx.y * blockDim.x;
    if ((t & 31) == 0)
#pragma unroll
        for (int q = 0; q < K; q++) sh[q][t >> 5] = v[q];
    __syncthreads();
    if (t == 0)
        for (int q = 0; q < K; q++) {
            double s = 0;
            for (int w = 0; w < BS / 32; w++) s += sh[q][w];
            out[q] = s;
        }
}

// sum of nblocks partials (stride apart, offset q) by the whole block, in a
// fixed order: thread t adds partials t, t + BS, ...; then a fixed tree
template <int BS>
__device__ __forceinline__ double block_final_sum(const double *part, int stride, int q,
                                                  int nblocks) {
    int t = threadIdx.x + threadIdx.y * blockDim.x;
    double v[1] = {0};
    for (int k = t; k < nblocks; k += BS) v[0] += part[(long long)k * stride + q];
    double out[1];
    block_sum<BS, 1>(v, out);
    __shared__ double res;
    if (t == 0) res = out[0];
    __syncthreads();
    double r = res;
    __syncthreads();
    return r;
}

// returns true in every thread of the last block to finish; the partials of
// all blocks are then visible
__device__ __forceinline__ bool last_block(unsigned int *ticket, unsigned int nblocks) {
    __shared__ bool last;
    int t = threadIdx.x + threadIdx.y * blockDim.x;
    __syncthreads();
    if (t == 0) {
        __threadfence();
        unsigned int prev = atomicAdd(ticket, 1u);
        last = prev == nblocks - 1;
    }
    __syncthreads();
    return last;
}

// k_surf: total surfactant sum (a+eps) psi + (chi+eps) C in FP64.
// mode 0: set the conserved total M0 (after initialisation);
// mode 1: end of a step: rescale factor M0/total (Sec. 2.2), SOR bookkeeping,
//         step counter, divergence check.
// rounds finished, from the counter the SOR loop leaves behind (an eager
// loop that stopped stores -(rounds) - 1000000)
__device__ __forceinline__ int sor_rounds_done(int e) { return e >= 0 ? e : -(e + 1000000); }

// k_surf: every thread sums a strip of SURF_STRIP cells along y in FP64;
// strips are added in FP64 across threads and blocks (one FP64 product pair
// a cell and step: negligible beside the step's FP32 work).
constexpr int SURF_STRIP = 4;

// block (bx, by) of a (gdx x .) grid of blockDim-shaped blocks
template <typename R, int BS>
__device__ __forceinline__ void surf2_block(const Inst<R> &I, int mode, int nblocks,
                                            int sweeps_per_round, int bx, int by, int gdx) {
    int x = bx * blockDim.x + threadIdx.x;
    // rows of the grid: y in 2D, (z, y) pairs in 3D (row index z ny + y)
    int y0 = (by * blockDim.y + threadIdx.y) * SURF_STRIP;
    const int rows = I.ny * I.nz;
    // after an odd number of blocked SOR rounds the solution is in psi2, C2
    const int rounds = sor_rounds_done(I.ctl->sor_exec);
    const bool alt = I.sor_pingpong && mode == 1 && ((rounds + I.sor_phase) & 1);
    const R *P = alt ? I.psi2 : I.psi;
    const R *Cc = alt ? I.C2 : I.C;
    // the strip's loads first (all in flight together), then the sum in
    // order: each product exact as hi + lo and the strip's sum compensated,
    // the total lbs_diagnostics forms in FP64 to rounding of the sum alone
    R va[SURF_STRIP], vp[SURF_STRIP], vb[SURF_STRIP], vc[SURF_STRIP];
#pragma unroll
    for (int k = 0; k < SURF_STRIP; k++) {
        const int y = y0 + k;
        va[k] = vp[k] = vb[k] = vc[k] = R(0);
        if (x < I.nx && y < rows) {
            const long long c = (long long)y * I.pitch + x;
            va[k] = I.a[c] + I.eps_w;
            vp[k] = P[c];
            vb[k] = I.chi[c] + I.eps_w;
            vc[k] = Cc[c];
        }
    }
    R hi = R(0), lo = R(0);
#pragma unroll
    for (int k = 0; k < SURF_STRIP; k++) {
        comp_add_prod(hi, lo, va[k], vp[k]);
        comp_add_prod(hi, lo, vb[k], vc[k]);
    }
    double v[1] = {double(hi) + double(lo)};
    int b = bx + by * gdx;
    block_sum<BS, 1>(v, I.part + b);
    if (!last_block(&I.ctl->ticket, nblocks)) return;
    const double tot = block_final_sum<BS>(I.part, 1, 0, nblocks);
    int t = threadIdx.x + threadIdx.y * blockDim.x;
    if (mode == 1) {  // the SOR convergence slots of the next solve start at zero
        unsigned long long *sw = &I.ctl->sweep[0][0];
        for (int k = t; k < KMAX_SWEEPS * 4; k += BS) sw[k] = 0ull;
    }
    if (t != 0) return;
    Ctl *ctl = I.ctl;
    ctl->ticket = 0;
    if (mode == 0) {
        ctl->M0 = tot;
        ctl->pre = tot;
        ctl->scale = 1.0;
        ctl->dscale = 0.0;
        ctl->dscale_f = 0.0f;
        return;
    }
    ctl->pre = tot;
    ctl->scale = tot > 0 ? ctl->M0 / tot : 1.0;
    ctl->dscale = ctl->scale - 1.0;
    ctl->dscale_f = float(ctl->dscale);
    if (!isfinite(tot)) {
        ctl->status |= ST_DIVERGED;
        ctl->dead = 1;
    }
    ctl->sor_iters = rounds * sweeps_per_round;
    ctl->sor_iters_parity = I.sor_pingpong ? ((rounds + I.sor_phase) & 1) : 0;
    ctl->sor_exec = 0;
    ctl->step += 1;
}

template <typename R, int BS>
__global__ void k_surf2(Inst<R> I, int mode, int nblocks, int sweeps_per_round) {
    pdl_trigger();
    surf2_block<R, BS>(I, mode, nblocks, sweeps_per_round, blockIdx.x, blockIdx.y, gridDim.x);
}

template <typename R>
__device__ __forceinline__ void scale2_cell(const Inst<R> &I, int x, int y, int z) {
    if (x >= I.nx || y >= I.ny) return;
    long long c = ((long long)z * I.ny + y) * I.pitch + x;
    // x (1 + d) with d = s - 1, rounded without bias
    // (rescale_one); the step counter has already advanced
    const double d = I.ctl->dscale;
    const float df = I.ctl->dscale_f;
    const long long n = I.ctl->step - 1;
    // the blocked SOR leaves its result in the second buffer after an odd
    // number of rounds
    const bool alt = I.ctl->sor_iters_parity != 0;
    const R p = alt ? I.psi2[c] : I.psi[c];
    const R q = alt ? I.C2[c] : I.C[c];
    I.psi[c] = rescale_one(p, d, df, rescale_key(c, 0, n));
    I.C[c] = rescale_one(q, d, df, rescale_key(c, 1, n));
}

template <typename R>
__global__ void k_scale2(Inst<R> I) {
    pdl_wait();
    scale2_cell(I, blockIdx.x * blockDim.x + threadIdx.x, blockIdx.y * blockDim.y + threadIdx.y, (int)blockIdx.z);
}

// step counter for runs without surfactant transport
template <typename R>
__global__ void k_tick(Inst<R> I) {
    if (threadIdx.x == 0 && blockIdx.x == 0) I.ctl->step += 1;
}

// ---------------------------------------------------------------------------
// Diagnostics (FP64): masses, total surfactant, indicator N = [rhoN >= 0]
// sums for U (Eqs. 33-34), centroid and second moments, interface psi stats.
// Q = 9 (D2Q9) or 19 (D3Q19); the grid's z index is the cell's z.
// ---------------------------------------------------------------------------
constexpr int NDIAG = 20;
constexpr int DIAG_STRIP = 16;  // cells per thread along y
template <typename R, typename P, int BS, int Q>
__global__ void k_diag(Inst<R> I, int nblocks) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y0 = (blockIdx.y * blockDim.y + threadIdx.y) * DIAG_STRIP;
    const int z = blockIdx.z;
    // 0 mR, 1 mB, 2 surf, 3 cnt, 4 sux, 5 suy, 6 sx, 7 sy, 8 sxx, 9 syy,
    // 10 psum, 11 pcnt, 12-14 (unused), 15 suz, 16 sz, 17 szz, 18 sxz, 19 sxy
    // (every thread a strip of DIAG_STRIP cells along y)
    double v[NDIAG] = {0};
    double pmin = 1e300, pmax = -1e300;
    const R *rhoN = mom_of_step(I, I.ctl->step).rN;
    double umax = 0.0;
    // the population set of the current step (the fused 2D step alternates
    // the two sets by the parity of the step counter)
    const bool odd = I.pop_pp && (I.ctl->step & 1);
    const void *pT = odd ? I.gT : I.fT, *pM = odd ? I.gM : I.fM;
    const R *pT0 = odd ? I.gT0 : I.fT0, *pM0 = odd ? I.gM0 : I.fM0;
    const uint8_t *pfl = odd ? I.gflag : I.flag;
    for (int kk = 0; kk < DIAG_STRIP && x < I.nx; kk++) {
        const int y = y0 + kk;
        if (y >= I.ny) break;
        long long c = ((long long)z * I.ny + y) * I.pitch + x;
        double rN = rhoN[c];
        // colour masses: the exact FP64 sums of the stored populations
        // (minority as stored, majority = shift + total deviation - minority)
        const int fl = pfl[c];
        double rmin = 0, rtot = 0;
        for (int i = 0; i < Q; i++) {
            rmin += double(ldq<R, P>(I, pM, pM0, i, c));
            rtot += double(i == 0 ? I.shift0[fl] : I.shift[i]) +
                    double(ldq<R, P>(I, pT, pT0, i, c));
        }
        v[0] += fl ? rtot - rmin : rmin;
        v[1] += fl ? rmin : rtot - rmin;
        v[2] += double(I.a[c] + I.eps_w) * double(I.psi[c]) +
                double(I.chi[c] + I.eps_w) * double(I.C[c]);
        // (velocities in the fields' own precision: FP64 storage gives FP64
        // diagnostics)
        const double ux = double(I.ux[c]), uy = double(I.uy[c]),
                     uz = Q == 19 ? double(I.uz[c]) : 0.0;
        if (rN >= 0) {
            v[3] += 1;
            v[4] += ux;
            v[5] += uy;
            v[6] += x;
            v[7] += y;
            v[8] += double(x) * x;
            v[9] += double(y) * y;
            v[15] += uz;
            v[16] += z;
            v[17] += double(z) * z;
            v[18] += double(x) * z;
            v[19] += double(x) * y;
        }
        if (fabs(rN) < 0.5) {
            double p = I.psi[c];
            v[10] += p;
            v[11] += 1;
            pmin = fmin(pmin, p);
            pmax = fmax(pmax, p);
        }
        umax = fmax(umax, sqrt(ux * ux + uy * uy + uz * uz));
    }
    int b = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    double s[NDIAG];
    block_sum<BS, NDIAG>(v, s);
    // min / max through a second pass on the same shared scheme
    double mm[4] = {-pmin, pmax, umax, 0};
    __shared__ double shm[3][BS / 32];
#pragma unroll
    for (int q = 0; q < 3; q++)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mm[q] = fmax(mm[q], __shfl_down_sync(0xffffffffu, mm[q], o));
    int t = threadIdx.x + threadIdx.y * blockDim.x;
    if ((t & 31) == 0)
        for (int q = 0; q < 3; q++) shm[q][t >> 5] = mm[q];
    __syncthreads();
    if (t == 0) {
        for (int q = 0; q < 3; q++) {
            double m = -1e300;
            for (int w = 0; w < BS / 32; w++) m = fmax(m, shm[q][w]);
            mm[q] = m;
        }
        for (int q = 0; q < NDIAG; q++) I.part[(long long)b * (NDIAG + 3) + q] = s[q];
        I.part[(long long)b * (NDIAG + 3) + NDIAG + 0] = mm[0];
        I.part[(long long)b * (NDIAG + 3) + NDIAG + 1] = mm[1];
        I.part[(long long)b * (NDIAG + 3) + NDIAG + 2] = mm[2];
    }
    if (!last_block(&I.ctl->ticket, nblocks)) return;
    // the NDIAG sums over the block partials in one pass (fixed order)
    double acc[NDIAG];
#pragma unroll
    for (int q = 0; q < NDIAG; q++) acc[q] = 0.0;
    for (int k = t; k < nblocks; k += BS)
#pragma unroll
        for (int q = 0; q < NDIAG; q++) acc[q] += I.part[(long long)k * (NDIAG + 3) + q];
    double tot[NDIAG];
    block_sum<BS, NDIAG>(acc, tot);
    if (t == 0)
        for (int q = 0; q < NDIAG; q++) I.ctl->diag[q] = tot[q];
    // the three maxima over the block partials, by the whole block
    double mx[3] = {-1e300, -1e300, -1e300};
    for (int k = t; k < nblocks; k += BS)
#pragma unroll
        for (int q = 0; q < 3; q++) mx[q] = fmax(mx[q], I.part[(long long)k * (NDIAG + 3) + NDIAG + q]);
#pragma unroll
    for (int q = 0; q < 3; q++)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx[q] = fmax(mx[q], __shfl_down_sync(0xffffffffu, mx[q], o));
    __syncthreads();
    if ((t & 31) == 0)
        for (int q = 0; q < 3; q++) shm[q][t >> 5] = mx[q];
    __syncthreads();
    if (t != 0) return;
    for (int q = 0; q < 3; q++) {
        double m = -1e300;
        for (int w = 0; w < BS / 32; w++) m = fmax(m, shm[q][w]);
        I.ctl->diag[NDIAG + q] = m;
    }
    I.ctl->ticket = 0;
}

// dense double copies of the intermediate fields of the current state
// (2D and 3D: the z components are null in 2D and exported as 0)
template <typename R>
__global__ void k_export_macro2(Inst<R> I, double *g, double *a, double *F, double *u) {
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= I.nx || y >= I.ny) return;
    const int z = blockIdx.z;
    long long c = ((long long)z * I.ny + y) * I.pitch + x;
    long long d = ((long long)z * I.ny + y) * I.nx + x;
    long long N = (long long)I.nx * I.ny * I.nz;
    g[d] = I.gx[c];
    g[N + d] = I.gy[c];
    g[2 * N + d] = I.gz ? double(I.gz[c]) : 0.0;
    a[d] = I.a[c];
    F[d] = I.Fx[c];
    F[N + d] = I.Fy[c];
    F[2 * N + d] = I.Fz ? double(I.Fz[c]) : 0.0;
    u[d] = I.ux[c];
    u[N + d] = I.uy[c];
    u[2 * N + d] = I.uz ? double(I.uz[c]) : 0.0;
}

// dense double copies of the macroscopic fields for the host
template <typename R>
__global__ void k_export2(Inst<R> I, double *rho, double *u, double *phi, double *psi,
                          double *C) {
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= I.nx || y >= I.ny) return;
    const int z = blockIdx.z;
    long long c = ((long long)z * I.ny + y) * I.pitch + x;
    long long d = ((long long)z * I.ny + y) * I.nx + x;
    long long N = (long long)I.nx * I.ny * I.nz;
    const MomSet<R> m = mom_of_step(I, I.ctl->step);
    rho[d] = double(m.rR[c]) + double(m.rB[c]);
    u[d] = I.ux[c];
    u[N + d] = I.uy[c];
    u[2 * N + d] = I.uz ? double(I.uz[c]) : 0.0;
    phi[d] = m.rN[c];
    psi[d] = I.psi[c];
    C[d] = I.C[c];
}

}  // namespace lbs
