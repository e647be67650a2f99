// lbs_k3d.cuh — D3Q19 kernels of the coupled LB-FD time step (arXiv
// 2311.15242; lattice of App. A, Eqs. 39-41).
//
// Same storage form and kernel sequence as the D2Q9 path (lbs_k2d.cuh):
// fT = total populations minus the rest state of the cell's majority phase,
// fM = populations of the cell's minority colour, a flag byte per cell.  The
// differences from 2D:
//   - the raw-moment matrix of Eq. 39 is not orthogonal; its inverse is the
//     closed form of lbs_d3q19.cuh;
//   - relaxation (Eq. 41): s = 1 on every row but the five second-order
//     shear rows 5-9, which take s_v of the mixture viscosity (Eq. 43);
//   - the correction of Eq. 40 acts on rows 4-6 with Q^k_a =
//     d_a{rho^k u_a [1 - 3 (c_s^k)^2]}, (c_s^k)^2 = (1 - alpha^k)/2;
//   - the interface weights, curvature, WENO fluxes and the diffusion
//     operator of Eq. 28 run over three axes (six faces);
//   - SOR: red-black half-sweeps as separate launches updating psi and C in
//     place (cells of one colour only read cells of the other colour when
//     every periodic axis has even length, which the host checks).
#pragma once

#include "lbs_d3q19.cuh"
#include "lbs_k2d.cuh"

namespace lbs {

template <typename R>
struct Mom3 {
    R rR, rB, drho, jx, jy, jz;
    R rm_s, rm_c, dr_s, dr_c;  // minority mass and drho as unevaluated sums s + c
};

template <typename R>
__device__ __forceinline__ Mom3<R> moments19(const Inst<R> &I, const R *fT, const R *fM,
                                            int flag) {
    Mom3<R> m{R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0)};
    CSum<R> rmc, drc;
#pragma unroll
    for (int i = 0; i < Q19; i++) {
        rmc.add(fM[i]);
        drc.add(fT[i]);
        if (ex19(i)) m.jx += R(ex19(i)) * fT[i];
        if (ey19(i)) m.jy += R(ey19(i)) * fT[i];
        if (ez19(i)) m.jz += R(ez19(i)) * fT[i];
    }
    const R rm = rmc.value();
    m.drho = drc.value();
    m.rm_s = rmc.s;
    m.rm_c = rmc.c;
    m.dr_s = drc.s;
    m.dr_c = drc.c;
    R rmaj = (I.rho_s[flag] - rm) + m.drho;
    m.rR = flag ? rmaj : rm;
    m.rB = flag ? rm : rmaj;
    return m;
}

template <typename R>
__device__ __forceinline__ void store_moments3(const Inst<R> &I, long long c, const R *fT,
                                               const R *fM, int flag) {
    Mom3<R> m = moments19(I, fT, fM, flag);
    I.rhoR[c] = m.rR;
    I.rhoB[c] = m.rB;
    I.rhoN[c] = colour_fn(I, m.rR, m.rB);
    I.jx[c] = m.jx;
    I.jy[c] = m.jy;
    I.jz[c] = m.jz;
}

#define LBS_CELL3                                               \
    const int x = blockIdx.x * blockDim.x + threadIdx.x;        \
    const int y = blockIdx.y * blockDim.y + threadIdx.y;        \
    const int z = blockIdx.z;                                   \
    if (x >= I.nx || y >= I.ny) return;                         \
    const long long c = cell3(I, x, y, z);

// initial populations f^k = M^{-1} m^{k,eq}(rho^k, u) (Eq. 40), in double
// precision and rounded once.  Inputs: dense double arrays [nz][ny][nx].
template <typename R, typename P>
__global__ void k_init3(Inst<R> I, const double *phi, const double *psi, const double *C,
                        const double *u) {
    LBS_CELL3
    const long long d = ((long long)z * I.ny + y) * I.nx + x;
    const long long N = (long long)I.nx * I.ny * I.nz;
    double ph = phi[d];
    ph = ph > 1.0 ? 1.0 : (ph < -1.0 ? -1.0 : ph);
    const double ux = u ? u[d] : 0.0, uy = u ? u[N + d] : 0.0, uz = u ? u[2 * N + d] : 0.0;
    double m[Q19], fR[Q19], fB[Q19];
    const double rR = double(I.rhoR0) * 0.5 * (1.0 + ph), rB = double(I.rhoB0) * 0.5 * (1.0 - ph);
    meq19<double>(rR, ux, uy, uz, double(I.alphaR), m);
    minv19<double>(m, fR);
    meq19<double>(rB, ux, uy, uz, double(I.alphaB), m);
    minv19<double>(m, fB);
    const int fl = (rR / double(I.rhoR0) <= rB / double(I.rhoB0)) ? 0 : 1;
    double tT = 0, tM = 0, sT = 0, sM = 0;
#pragma unroll
    for (int i = 0; i < Q19; i++) {
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

template <typename R, typename P>
__global__ void k_moments3(Inst<R> I) {
    LBS_CELL3
    R fT[Q19], fM[Q19];
#pragma unroll
    for (int i = 0; i < Q19; i++) {
        fT[i] = ldq<R, P>(I, I.fT, I.fT0, i, c);
        fM[i] = ldq<R, P>(I, I.fM, I.fM0, i, c);
    }
    store_moments3(I, c, fT, fM, I.flag[c]);
}

// colour gradient by the isotropic stencil over the 18 neighbours, from the
// colour fraction that is small on the cell's side (see k_grad2)
template <typename R>
__global__ void k_grad3(Inst<R> I, int guess = 1) {
    LBS_CELL3
    const bool blue_side = I.rhoN[c] <= R(0);
    const Ax X = make_ax(x, I.nx, I.wall[0], 1), Y = make_ax(y, I.ny, I.wall[1], 2),
             Z = make_ax(z, I.nz, I.wall[2], 4);
    R gx = R(0), gy = R(0), gz = R(0);
#pragma unroll
    for (int i = 1; i < Q19; i++) {
        int refl, sx, sy, sz;
        long long j = nbx3(I, X, Y, Z, ex19(i), ey19(i), ez19(i), refl, sx, sy, sz);
        R v = w19<R>(i) * frac(I, j, blue_side);
        if (ex19(i)) gx += R(ex19(i)) * v;
        if (ey19(i)) gy += R(ey19(i)) * v;
        if (ez19(i)) gz += R(ez19(i)) * v;
    }
    const R f = blue_side ? R(6) : R(-6);  // 2 / c_s^2
    gx *= f;
    gy *= f;
    gz *= f;
    I.gx[c] = gx;
    I.gy[c] = gy;
    I.gz[c] = gz;
    I.a[c] = sqrt(gx * gx + gy * gy + gz * gz);
    I.chi[c] = R(2) * frac(I, c, false);
    if (guess) sor_guess(I, c);
}

// normal, curvature (Eq. 7), grad psi, sigma (Eq. 8), interfacial force
// (Eq. 9) plus buoyancy, velocity (Eq. 10)
template <typename R>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 5 : 2) k_force3(Inst<R> I) {
    LBS_CELL3
    const R e2 = I.eps_n * I.eps_n;
    const Ax X = make_ax(x, I.nx, I.wall[0], 1), Y = make_ax(y, I.ny, I.wall[1], 2),
             Z = make_ax(z, I.nz, I.wall[2], 4);
    R divn = R(0), dpx = R(0), dpy = R(0), dpz = R(0);
#pragma unroll
    for (int i = 1; i < Q19; i++) {
        int refl, sx, sy, sz;
        long long j = nbx3(I, X, Y, Z, ex19(i), ey19(i), ez19(i), refl, sx, sy, sz);
        R gx = I.gx[j], gy = I.gy[j], gz = I.gz[j];
        if (refl & 1) gx = -gx;  // normal component mirrored with a sign change
        if (refl & 2) gy = -gy;
        if (refl & 4) gz = -gz;
        const R inv = frsq(gx * gx + gy * gy + gz * gz + e2);
        R s = R(0);
        if (ex19(i)) s += R(ex19(i)) * gx;
        if (ey19(i)) s += R(ey19(i)) * gy;
        if (ez19(i)) s += R(ez19(i)) * gz;
        divn -= w19<R>(i) * s * inv;
        const R p = w19<R>(i) * I.psi[j];
        if (ex19(i)) dpx += R(ex19(i)) * p;
        if (ey19(i)) dpy += R(ey19(i)) * p;
        if (ez19(i)) dpz += R(ez19(i)) * p;
    }
    const R kappa = -R(3) * divn;
    dpx *= R(3);
    dpy *= R(3);
    dpz *= R(3);
    const R gx = I.gx[c], gy = I.gy[c], gz = I.gz[c], a = I.a[c];
    R sigma, mco, Fx, Fy, Fz;
    if (eos(I, I.psi[c], sigma, mco)) {
        const R inv = frsq(gx * gx + gy * gy + gz * gz + e2);
        const R nx = -gx * inv, ny = -gy * inv, nz = -gz * inv;
        const R ndp = nx * dpx + ny * dpy + nz * dpz;
        Fx = -R(0.5) * sigma * kappa * gx - R(0.5) * a * mco * (dpx - ndp * nx);
        Fy = -R(0.5) * sigma * kappa * gy - R(0.5) * a * mco * (dpy - ndp * ny);
        Fz = -R(0.5) * sigma * kappa * gz - R(0.5) * a * mco * (dpz - ndp * nz);
    } else {
        Fx = -R(0.5) * I.sigma_min * kappa * gx;
        Fy = -R(0.5) * I.sigma_min * kappa * gy;
        Fz = -R(0.5) * I.sigma_min * kappa * gz;
    }
    const R rR = I.rhoR[c], rB = I.rhoB[c];
    const R rho = rR + rB;
    const R drb = rR + (rB - I.rhoB0);
    Fx += drb * I.g[0];
    Fy += drb * I.g[1];
    Fz += drb * I.g[2];
    I.Fx[c] = Fx;
    I.Fy[c] = Fy;
    I.Fz[c] = Fz;
    const R irho = fdiv(R(1), rho);
    I.ux[c] = (I.jx[c] + R(0.5) * Fx) * irho;
    I.uy[c] = (I.jy[c] + R(0.5) * Fy) * irho;
    I.uz[c] = (I.jz[c] + R(0.5) * Fz) * irho;
}

// explicit surfactant terms (Eqs. 22-27) and Crank-Nicolson right-hand sides
// with the six-face operator of Eq. 28; Sout / Bout: export only (see k_fd2)
template <typename R>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 4 : 2)
    k_fd3(Inst<R> I, double *Sout = nullptr, double *Bout = nullptr) {
    LBS_CELL3
    const R u[3] = {I.ux[c], I.uy[c], I.uz[c]};
    const R *uax[3] = {I.ux, I.uy, I.uz};
    const Ax X = make_ax(x, I.nx, I.wall[0], 1), Y = make_ax(y, I.ny, I.wall[1], 2),
             Z = make_ax(z, I.nz, I.wall[2], 4);
    R divP = R(0), divC = R(0);
#pragma unroll
    for (int ax = 0; ax < 3; ax++) {
        R Pl[5], Cl[5];
#pragma unroll
        for (int k = -2; k <= 2; k++) {
            int refl, sx, sy, sz;
            long long j = nbx3(I, X, Y, Z, ax == 0 ? k : 0, ax == 1 ? k : 0, ax == 2 ? k : 0,
                               refl, sx, sy, sz);
            const R sgn = (refl & (1 << ax)) ? R(-1) : R(1);
            const R uj = uax[ax][j];
            Pl[k + 2] = sgn * I.psi[j] * I.a[j] * uj;
            Cl[k + 2] = sgn * I.C[j] * I.chi[j] * uj;
        }
        divP += upwind(Pl + 2, u[ax]);
        divC += upwind(Cl + 2, u[ax]);
    }
    const R psi = I.psi[c], Cc = I.C[c], a = I.a[c];
    const R jj = I.source == 1 ? I.ra * I.psi_inf * Cc
                               : I.ra * Cc * (I.psi_inf - psi) - I.rd * psi;
    const R S = -divP + a * jj;
    const R B = -divC - a * jj;
    if (Sout) {
        const long long d = ((long long)z * I.ny + y) * I.nx + x;
        Sout[d] = S;
        Bout[d] = B;
        return;
    }
    const R wp = a + I.eps_w, wc = I.chi[c] + I.eps_w;
    R Lp = R(0), Lc = R(0);
#pragma unroll
    for (int f = 0; f < 6; f++) {
        const int s = (f & 1) ? 1 : -1, ax = f >> 1;
        int refl, sx, sy, sz;
        long long j2 = nbx3(I, X, Y, Z, ax == 0 ? s : 0, ax == 1 ? s : 0, ax == 2 ? s : 0,
                            refl, sx, sy, sz);
        if (refl) continue;
        Lp += R(0.5) * (wp + (I.a[j2] + I.eps_w)) * (I.psi[j2] - psi);
        Lc += R(0.5) * (wc + (I.chi[j2] + I.eps_w)) * (I.C[j2] - Cc);
    }
    const bool first = I.ctl->step == 0;
    const R Sp = I.S[c], Bp = I.B[c];
    const R abS = first ? S : R(1.5) * S - R(0.5) * Sp;
    const R abB = first ? B : R(1.5) * B - R(0.5) * Bp;
    I.rpsi[c] = wp * psi + R(0.5) * I.Ds * Lp + abS;
    I.rC[c] = wc * Cc + R(0.5) * I.Db * Lc + abB;
    I.S[c] = S;
    I.B[c] = B;
}

// ---------------------------------------------------------------------------
// k_collide3: MRT collision in raw-moment space (Eqs. 1-4, 39-41, 43) on the
// shifted total populations, then recolouring (Eqs. 11-12).
//   m - m^eq per row, with P = sum_k rho^k (c_s^k)^2, dP = P minus the
//   pressure of the shift (the pure majority phase at rest):
//     row 0: 0;   rows 1-3: -F/2 exactly (u carries the half force)
//     row 4: mT4 - 3 dP - rho u^2
//     rows 5-9: mT - rho (2ux^2-uy^2-uz^2, uy^2-uz^2, ux uy, ux uz, uy uz)
//     rows 10-15: mT - P (uy, ux, uz, ux, uz, uy)
//     rows 16-18: mT - dP/3 - rho (ux^2+uy^2-uz^2, ux^2+uz^2-uy^2,
//                                  uy^2+uz^2-ux^2) / 6
//   forcing moments of Eq. 4 for D3Q19 in closed form (isotropy of the
//   weights to fourth order; rows 16-18 from the sixth-order sums):
//     F0 = 0, F1-3 = F, F4 = 2 u.F, F5 = 4uxFx - 2uyFy - 2uzFz,
//     F6 = 2uyFy - 2uzFz, F7 = uxFy + uyFx, F8 = uxFz + uzFx, F9 = uyFz + uzFy,
//     F10-15 = (Fy, Fx, Fz, Fx, Fz, Fy)/3,
//     F16 = uxFx + uyFy - u.F/3, F17 = uxFx + uzFz - u.F/3, F18 = uyFy + uzFz - u.F/3
//   change of the moments: dm = -S (m - m^eq) + (1 - S/2)(C + F); rows 1-3
//   then give F.
// ---------------------------------------------------------------------------
template <typename R, typename P>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 3 : 2) k_collide3(Inst<R> I) {
    LBS_CELL3
    R fT[Q19], fM[Q19];
    const int fl = I.flag[c];
#pragma unroll
    for (int i = 0; i < Q19; i++) {
        fT[i] = ldq<R, P>(I, I.fT, I.fT0, i, c);
        fM[i] = ldq<R, P>(I, I.fM, I.fM0, i, c);
    }
    const Mom3<R> mo = moments19(I, fT, fM, fl);
    const R rR = mo.rR, rB = mo.rB;
    const R rmin = fl ? rB : rR;
    const R devmaj = I.dsh[fl] + (mo.drho - rmin);
    const R rho = rR + rB;
    const R ux = I.ux[c], uy = I.uy[c], uz = I.uz[c];
    const R Fx = I.Fx[c], Fy = I.Fy[c], Fz = I.Fz[c];

    // d_a(rho^k u_a), isotropic stencil, ghost velocities at walls
    R dR[3] = {R(0), R(0), R(0)}, dB[3] = {R(0), R(0), R(0)};
    const Ax X = make_ax(x, I.nx, I.wall[0], 1), Y = make_ax(y, I.ny, I.wall[1], 2),
             Z = make_ax(z, I.nz, I.wall[2], 4);
#pragma unroll
    for (int i = 1; i < Q19; i++) {
        int refl, sx, sy, sz;
        long long j = nbx3(I, X, Y, Z, ex19(i), ey19(i), ez19(i), refl, sx, sy, sz);
        R vx = I.ux[j], vy = I.uy[j], vz = I.uz[j];
        ghost_u3(I, refl, sx, sy, sz, vx, vy, vz);
        const R r1 = w19<R>(i) * I.rhoR[j], r2 = w19<R>(i) * I.rhoB[j];
        if (ex19(i)) {
            dR[0] += R(ex19(i)) * r1 * vx;
            dB[0] += R(ex19(i)) * r2 * vx;
        }
        if (ey19(i)) {
            dR[1] += R(ey19(i)) * r1 * vy;
            dB[1] += R(ey19(i)) * r2 * vy;
        }
        if (ez19(i)) {
            dR[2] += R(ez19(i)) * r1 * vz;
            dB[2] += R(ez19(i)) * r2 * vz;
        }
    }
    const R cR = R(1) - R(1.5) * (R(1) - I.alphaR), cB = R(1) - R(1.5) * (R(1) - I.alphaB);
    const R Qx = R(3) * (cR * dR[0] + cB * dB[0]);
    const R Qy = R(3) * (cR * dR[1] + cB * dB[1]);
    const R Qz = R(3) * (cR * dR[2] + cB * dB[2]);

    // moments of the shifted total populations (rows 4-18)
    R mT[Q19];
#pragma unroll
    for (int j = 4; j < Q19; j++) {
        R s = R(0);
#pragma unroll
        for (int i = 0; i < Q19; i++)
            if (m19(j, i) != 0) s += R(m19(j, i)) * fT[i];
        mT[j] = s;
    }
    const R Pk = rR * I.cs2R + rB * I.cs2B;
    const R dP = fl == 0 ? devmaj * I.cs2B + rR * I.cs2R : devmaj * I.cs2R + rB * I.cs2B;
    const R xx = ux * ux, yy = uy * uy, zz = uz * uz, u2 = xx + yy + zz;
    R neq[Q19];
    neq[4] = mT[4] - R(3) * dP - rho * u2 + I.mcor1[fl];
    neq[5] = mT[5] - rho * (R(2) * xx - yy - zz);
    neq[6] = mT[6] - rho * (yy - zz);
    neq[7] = mT[7] - rho * ux * uy;
    neq[8] = mT[8] - rho * ux * uz;
    neq[9] = mT[9] - rho * uy * uz;
    neq[10] = mT[10] - Pk * uy;
    neq[11] = mT[11] - Pk * ux;
    neq[12] = mT[12] - Pk * uz;
    neq[13] = mT[13] - Pk * ux;
    neq[14] = mT[14] - Pk * uz;
    neq[15] = mT[15] - Pk * uy;
    const R d3 = dP / R(3) - I.mcor2[fl];
    neq[16] = mT[16] - d3 - rho * (xx + yy - zz) / R(6);
    neq[17] = mT[17] - d3 - rho * (xx + zz - yy) / R(6);
    neq[18] = mT[18] - d3 - rho * (yy + zz - xx) / R(6);

    // s_v from the mixture viscosity (Eq. 43)
    const R rN = colour_fn(I, rR, rB);
    const R inv_mu = (R(1) + rN) * I.inv_2muR + (R(1) - rN) * I.inv_2muB;
    const R sv = fdiv(R(1), R(0.5) + fdiv(R(1), inv_mu * Pk));
    const R uF = ux * Fx + uy * Fy + uz * Fz;
    const R xF = ux * Fx, yF = uy * Fy, zF = uz * Fz;
    R dm[Q19];
    dm[0] = R(0);
    dm[1] = Fx;
    dm[2] = Fy;
    dm[3] = Fz;
    dm[4] = -neq[4] + R(0.5) * ((Qx + Qy + Qz) + R(2) * uF);
    const R hv = R(1) - R(0.5) * sv;
    dm[5] = -sv * neq[5] + hv * ((R(2) * Qx - Qy - Qz) + (R(4) * xF - R(2) * yF - R(2) * zF));
    dm[6] = -sv * neq[6] + hv * ((Qy - Qz) + (R(2) * yF - R(2) * zF));
    dm[7] = -sv * neq[7] + hv * (ux * Fy + uy * Fx);
    dm[8] = -sv * neq[8] + hv * (ux * Fz + uz * Fx);
    dm[9] = -sv * neq[9] + hv * (uy * Fz + uz * Fy);
    const R t3 = R(0.5) / R(3);
    dm[10] = -neq[10] + t3 * Fy;
    dm[11] = -neq[11] + t3 * Fx;
    dm[12] = -neq[12] + t3 * Fz;
    dm[13] = -neq[13] + t3 * Fx;
    dm[14] = -neq[14] + t3 * Fz;
    dm[15] = -neq[15] + t3 * Fy;
    const R u3 = uF / R(3);
    dm[16] = -neq[16] + R(0.5) * (xF + yF - u3);
    dm[17] = -neq[17] + R(0.5) * (xF + zF - u3);
    dm[18] = -neq[18] + R(0.5) * (yF + zF - u3);
    R df[Q19];
    minv19<R>(dm, df);

    R post[Q19];
    CSum<R> rdc;
#pragma unroll
    for (int i = 0; i < Q19; i++) {
        post[i] = fT[i] + df[i];
        rdc.add(shift_of(I, i, fl) + post[i]);
    }
    const R rdag = rdc.value();
    // recolouring: segregation weight f_i^eq(rho, 0)/rho = w_i 3 P / rho for
    // the moving directions (the rest equilibrium of Eq. 40: rho - 2P at rest,
    // P/6 on the axes, P/12 on the diagonals)
    const R ggx = I.gx[c], ggy = I.gy[c], ggz = I.gz[c];
    const R seg = I.beta * rR * rB * R(3) * Pk *
                  frsq(ggx * ggx + ggy * ggy + ggz * ggz + I.eps_n * I.eps_n) *
                  fdiv(R(1), rho * rho);
    const R fr = fdiv(rmin, rdag);
    const R sg = fl ? R(-1) : R(1);
    // moving populations as stored; the rest populations close the cell's
    // total and minority mass on the pre-collision values (see k_collide2)
    CSum<R> sT, sM;
    const unsigned int rk = rest_key(c, rest_salt(0, I.ctl->step)), rs = pop_seed(rk);
#pragma unroll
    for (int i = 1; i < Q19; i++) {
        R eg = R(0);
        if (ex19(i)) eg += R(ex19(i)) * ggx;
        if (ey19(i)) eg += R(ey19(i)) * ggy;
        if (ez19(i)) eg += R(ez19(i)) * ggz;
        const R segi = seg * w19<R>(i) * eg;
        sT.add(stq_r<R, P>(I, I.gT, i, c, post[i], pop_r(rs, 2 * i)));
        sM.add(stq_r<R, P>(I, I.gM, i, c, fr * (I.shift[i] + post[i]) + sg * segi,
                           pop_r(rs, 2 * i + 1)));
    }
    I.gT0[c] = rest_close(mo.dr_s, mo.dr_c, sT.s, sT.c, R(0), rest_u(rk, 0));
    I.gM0[c] = rest_close(mo.rm_s, mo.rm_c, sM.s, sM.c, R(0), rest_u(rk, 1));
    I.gflag[c] = (uint8_t)fl;
}

// streaming (Eq. 13, pull), half-way bounce-back with moving walls, moments
// at t+1 (see k_stream2).  MIRROR: the grid has mirror planes (a separate
// instantiation, so that grids without them keep the plain direction choice)
template <typename R, typename P, bool MIRROR>
__global__ void __launch_bounds__(256, 3) k_stream3(Inst<R> I) {
    LBS_CELL3
    const int flc = I.gflag[c];
    const Ax X = make_ax(x, I.nx, I.wall[0], 1), Y = make_ax(y, I.ny, I.wall[1], 2),
             Z = make_ax(z, I.nz, I.wall[2], 4);
    // 1. the streamed (total, minority) pairs as stored at their sources;
    //    a link that crosses a wall reflects the cell's own opposite
    //    population; slow: bit i set where the source's flag differs from the
    //    cell's or the link crosses a moving wall
    R t[Q19], m[Q19];
    unsigned slow = 0, fbits = 0;
    // (branch-free: a reflected link reads the cell's own opposite
    // population, so that every load of the loop can be in flight at once)
#pragma unroll
    for (int i = 0; i < Q19; i++) {
        int refl, sx, sy, sz;
        const long long j = nbx3(I, X, Y, Z, -ex19(i), -ey19(i), -ez19(i), refl, sx, sy, sz);
        if (i == 0) {
            t[0] = I.gT0[c];
            m[0] = I.gM0[c];
            continue;
        }
        const int bb = refl & I.bbmask;  // mirror planes: the mirrored source
        const long long src = bb ? c : j;
        const int dir = bb ? opp19(i) : (MIRROR ? mir19(i, refl) : i);
        const long long k = (long long)dir * I.plane + src;
        t[i] = ldp<R, P>(I, I.gT, k);
        m[i] = ldp<R, P>(I, I.gM, k);
        const int fj = I.gflag[src];
        fbits |= (unsigned)fj << i;
        // (a static wall returns the cell's own opposite population unchanged:
        // the fast path's plain move; a moving wall adds its momentum term)
        if (fj != flc || (bb & I.mvmask)) slow |= 1u << i;
    }
    fbits |= (unsigned)flc;  // (i = 0: the cell's own flag)
    // 2. fast path: every population moves unchanged; the cell keeps its
    //    flag unless its minority colour has become the majority
    if (!slow) {
        CSum<R> tot, mn;
        R jx = R(0), jy = R(0), jz = R(0);
#pragma unroll
        for (int i = 0; i < Q19; i++) {
            tot.add(t[i]);
            mn.add(m[i]);
            if (ex19(i)) jx += R(ex19(i)) * t[i];
            if (ey19(i)) jy += R(ey19(i)) * t[i];
            if (ez19(i)) jz += R(ez19(i)) * t[i];
        }
        const R rmin = mn.value(), rmaj = (I.rho_s[flc] - rmin) + tot.value();
        const R rR = flc ? rmaj : rmin, rB = flc ? rmin : rmaj;
        if (minority(I, rR, rB) == flc) {
#pragma unroll
            for (int i = 1; i < Q19; i++) {
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
            I.jz[c] = jz;
            return;
        }
    }
    // 3. general path: colours re-split where the flags differ, moving-wall
    //    terms added; every value carried as hi + lo (TwoSum errors), and
    //    the rest populations close the cell's masses exactly
    const R rRc = I.rhoR[c], rBc = I.rhoB[c];
    R fR[Q19], fB[Q19];
    R loT = R(0), loR = R(0), loB = R(0);
#pragma unroll
    for (int i = 0; i < Q19; i++) {
        const int fj = (fbits >> i) & 1;
        R tlo = R(0), mlo = R(0);
        R sh = shift_of(I, i, fj);
        if ((slow >> i) & 1) {
            int refl, sx, sy, sz;
            nbx3(I, X, Y, Z, -ex19(i), -ey19(i), -ez19(i), refl, sx, sy, sz);
            refl &= I.bbmask;  // (mirror planes reflect without a wall term)
            if (refl) {
                R uw[3] = {R(0), R(0), R(0)};
                int nw = 0;
                const int side[3] = {sx, sy, sz};
#pragma unroll
                for (int a = 0; a < 3; a++) {
                    if (!(refl & (1 << a))) continue;
                    const R *w = side[a] < 0 ? I.uw_lo[a] : I.uw_hi[a];
                    uw[0] += w[0];
                    uw[1] += w[1];
                    uw[2] += w[2];
                    nw++;
                }
                const R eu =
                    (R(ex19(i)) * uw[0] + R(ey19(i)) * uw[1] + R(ez19(i)) * uw[2]) / R(nw);
                const R mw = R(2) * w19<R>(i) * eu * R(3);
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
    for (int i = 0; i < Q19; i++) {
        rR += fR[i];
        rB += fB[i];
    }
    const int fl = minority(I, rR, rB);
    if (fl != flc) {
        R d1, d2;
        const R d = two_sum(I.shift0[flc], -I.shift0[fl], d1);
        t[0] = two_sum(d, t[0], d2);
        loT += d1 + d2;
    }
    R fT[Q19], fM[Q19];
    CSum<R> gT, gM, sT, sM;
    const R loM = fl ? loB : loR;
    const unsigned int rk = rest_key(c, rest_salt(1, I.ctl->step)), rs = pop_seed(rk);
#pragma unroll
    for (int i = 0; i < Q19; i++) {
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
    store_moments3(I, c, fT, fM, fl);
}

// block maxima of a half-sweep -> the round's slot; after the black
// half-sweep the last block decides whether another round runs
template <typename R, int BS>
__device__ __forceinline__ void sor3_finish(const Inst<R> &I, int round, int colour, R v[4],
                                            cudaGraphConditionalHandle loop, int max_rounds,
                                            int eager_round) {
    __shared__ R sh[4][BS / 32];
    const int t = threadIdx.x + threadIdx.y * blockDim.x;
#pragma unroll
    for (int q = 0; q < 4; q++)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[q] = fmax(v[q], __shfl_down_sync(0xffffffffu, v[q], o));
    if ((t & 31) == 0)
        for (int q = 0; q < 4; q++) sh[q][t >> 5] = v[q];
    __syncthreads();
    if (t == 0)
        for (int q = 0; q < 4; q++) {
            R m = R(0);
            for (int w = 0; w < BS / 32; w++) m = fmax(m, sh[q][w]);
            atomic_max_pos(&I.ctl->sweep[round][q], double(m));
        }
    if (colour == 0) return;
    const unsigned int nb = gridDim.x * gridDim.y * gridDim.z;
    if (!last_block(&I.ctl->sor_ticket, nb)) return;
    if (t != 0) return;
    Ctl *ctl = I.ctl;
    ctl->sor_ticket = 0;
    const bool conv = round_converged<R>(ctl, round, double(I.sor_tol));
    const bool stop = conv || round + 1 >= max_rounds;
    if (stop && !conv) ctl->status |= ST_NOCONV;
    if (eager_round < 0) {
        ctl->sor_exec = round + 1;
        if (stop) cudaGraphSetConditional(loop, 0);
    } else {
        ctl->sor_exec = stop ? -(round + 1) - 1000000 : round + 1;
    }
}

// ---------------------------------------------------------------------------
// k_sor_rb3: one half-sweep of red-black SOR (omega of Sec. 2.2) for
// (w - h L_w) x = rhs on psi and C, updating the cells of one colour
// ((x + y + z) mod 2) in place.  Thread (tx, y, z) takes the cell
// x = 2 tx + ((y + z + colour) mod 2).  Both half-sweeps fold their largest
// update and value into the round's slot; the black launch's last block
// decides whether another round (sweep) runs.
// ---------------------------------------------------------------------------
template <typename R, int BS>
__global__ void __launch_bounds__(BS)
    k_sor_rb3(Inst<R> I, int colour, cudaGraphConditionalHandle loop, int max_rounds,
              int eager_round) {
    if (eager_round > 0 && I.ctl->sor_exec < eager_round) return;  // loop already ended
    const int round = I.ctl->sor_exec;
    const int tx = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    const int x = 2 * tx + ((y + z + colour) & 1);
    R v[4] = {R(0), R(0), R(0), R(0)};
    if (x < I.nx && y < I.ny) {
        const long long c = cell3(I, x, y, z);
        const R hp = R(0.5) * I.Ds, hc = R(0.5) * I.Db;
        const R wp = I.a[c] + I.eps_w, wc = I.chi[c] + I.eps_w;
        R dp = wp, dc = wc, op = I.rpsi[c], oc = I.rC[c];
        const Ax X = make_ax(x, I.nx, I.wall[0], 1), Y = make_ax(y, I.ny, I.wall[1], 2),
                 Z = make_ax(z, I.nz, I.wall[2], 4);
#pragma unroll
        for (int f = 0; f < 6; f++) {
            const int s = (f & 1) ? 1 : -1, ax = f >> 1;
            int refl, sx, sy, sz;
            long long j = nbx3(I, X, Y, Z, ax == 0 ? s : 0, ax == 1 ? s : 0, ax == 2 ? s : 0,
                               refl, sx, sy, sz);
            if (refl) continue;  // no flux through a wall
            const R fp = hp * (R(0.5) * (wp + (I.a[j] + I.eps_w)));
            const R fc = hc * (R(0.5) * (wc + (I.chi[j] + I.eps_w)));
            dp += fp;
            dc += fc;
            op += fp * I.psi[j];
            oc += fc * I.C[j];
        }
        const R p0 = I.psi[c], c0 = I.C[c];
        const R d1 = I.omega * (fdiv(op, dp) - p0), d2 = I.omega * (fdiv(oc, dc) - c0);
        const R p1 = p0 + d1, c1 = c0 + d2;
        I.psi[c] = p1;
        I.C[c] = c1;
        v[0] = fabs(d1);
        v[1] = fabs(d2);
        v[2] = fabs(p1);
        v[3] = fabs(c1);
    }
    sor3_finish<R, BS>(I, round, colour, v, loop, max_rounds, eager_round);
}

// ---------------------------------------------------------------------------
// k_sor_cm3: the half-sweep of k_sor_rb3 (same faces, summed in the same
// order) by column marching.  Lane l of a warp owns the cell pair
// x0 = 2 (32 bx + l), x0 + 1 of row y (a warp is one row) and marches z over
// a chunk of ZC planes; on plane z it updates the pair's cell of the current
// colour, x0 + k with k = (colour + y + z) mod 2.  The pair's psi, C, a and
// chi on planes z - 1, z and z + 1 stay in registers (plane z + 2 is loaded
// a step ahead).  The x-neighbour outside the pair is the adjacent lane's
// pair: k is the same for the whole warp, so all lanes take the same side;
// only the warp's and the domain's end lanes load it.  The y-neighbours and
// the right-hand sides are loaded.  The cells a half-sweep reads (the other
// colour) and writes (its colour) are disjoint, so no thread reads a value
// another thread writes.
// ---------------------------------------------------------------------------
template <typename R>
struct Pair4 {  // psi, C, a, chi of a cell pair on one plane
    R p0, p1, c0, c1, a0, a1, x0, x1;
    bool wall;  // the plane lies beyond a wall
};

template <typename R>
__device__ __forceinline__ void load_pair3(const Inst<R> &I, int x0, bool act, int y, int zz,
                                           Pair4<R> &q) {
    int refl = 0, side;
    const int z = map_axis(zz, I.nz, I.wall[2], 4, refl, side);
    q.wall = refl != 0;
    if (!act || refl) {
        q.p0 = q.p1 = q.c0 = q.c1 = q.a0 = q.a1 = q.x0 = q.x1 = R(0);
        return;
    }
    using V = typename Vec2<R>::T;
    const long long c = cell3(I, x0, y, z);  // even: x0 and the pitch are even
    const V p = *(const V *)&I.psi[c], cc = *(const V *)&I.C[c];
    const V a = *(const V *)&I.a[c], x = *(const V *)&I.chi[c];
    q.p0 = p.x;
    q.p1 = p.y;
    q.c0 = cc.x;
    q.c1 = cc.y;
    q.a0 = a.x;
    q.a1 = a.y;
    q.x0 = x.x;
    q.x1 = x.y;
}

// right-hand sides and the y-neighbours' a, chi, psi, C of the cell a
// column-marching thread updates on one plane (zero where not needed)
template <typename R>
struct Nb3 {
    R rp, rc, am, xm, pm, cm, ap, xp, pp, cp;
};
template <typename R>
__device__ __forceinline__ void load_nb3(const Inst<R> &I, bool on, int xu, int y, int ym,
                                         int yp, bool rym, bool ryp, int z, Nb3<R> &n) {
    n.rp = n.rc = n.am = n.xm = n.pm = n.cm = n.ap = n.xp = n.pp = n.cp = R(0);
    if (!on) return;
    const long long c = cell3(I, xu, y, z);
    n.rp = I.rpsi[c];
    n.rc = I.rC[c];
    if (!rym) {
        const long long j = cell3(I, xu, ym, z);
        n.am = I.a[j];
        n.xm = I.chi[j];
        n.pm = I.psi[j];
        n.cm = I.C[j];
    }
    if (!ryp) {
        const long long j = cell3(I, xu, yp, z);
        n.ap = I.a[j];
        n.xp = I.chi[j];
        n.pp = I.psi[j];
        n.cp = I.C[j];
    }
}

template <typename R, int BS, int ZC>
__global__ void __launch_bounds__(BS)
    k_sor_cm3(Inst<R> I, int colour, cudaGraphConditionalHandle loop, int max_rounds,
              int eager_round) {
    if (eager_round > 0 && I.ctl->sor_exec < eager_round) return;  // loop already ended
    const int round = I.ctl->sor_exec;
    const int lane = threadIdx.x;  // blockDim.x == 32
    const int x0 = 2 * (blockIdx.x * 32 + lane);
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int zs = blockIdx.z * ZC, ze = min(zs + ZC, I.nz);
    const bool act = x0 < I.nx;
    R v[4] = {R(0), R(0), R(0), R(0)};
    if (y < I.ny) {  // (the whole warp)
        const R hp = R(0.5) * I.Ds, hc = R(0.5) * I.Db;
        int side;
        // neighbours along y, the pair's partner beyond a wall (odd nx), and
        // the x-neighbours outside the pair: x0 - 1 (k = 0), x0 + 2 (k = 1)
        int rym = 0, ryp = 0, rpart = 0, rxa = 0, rxb = 0;
        const int ym = map_axis(y - 1, I.ny, I.wall[1], 2, rym, side);
        const int yp = map_axis(y + 1, I.ny, I.wall[1], 2, ryp, side);
        map_axis(x0 + 1, I.nx, I.wall[0], 1, rpart, side);
        const int xa = map_axis(x0 - 1, I.nx, I.wall[0], 1, rxa, side);
        const int xb = map_axis(x0 + 2, I.nx, I.wall[0], 1, rxb, side);
        // the adjacent lane holds that neighbour when it is inside the domain
        const bool sha = lane > 0 && x0 >= 2, shb = lane < 31 && x0 + 2 < I.nx;
        Pair4<R> Pm, P0, Pp, Pn;
        load_pair3(I, x0, act, y, zs - 1, Pm);
        load_pair3(I, x0, act, y, zs, P0);
        load_pair3(I, x0, act, y, zs + 1, Pp);
        // the loads of a plane's own cell and y-neighbours go out one plane
        // ahead of its update (cells of the other colour and right-hand
        // sides: nothing this half-sweep writes)
        Nb3<R> nb;
        {
            const int xu = x0 + ((colour + y + zs) & 1);
            load_nb3(I, act && xu < I.nx, xu, y, ym, yp, rym, ryp, zs, nb);
        }
        for (int z = zs; z < ze; z++) {
            if (z + 2 <= ze) load_pair3(I, x0, act, y, z + 2, Pn);
            const int k = (colour + y + z) & 1;
            const Nb3<R> cur = nb;
            if (z + 1 < ze) {
                const int xn = x0 + 1 - k;
                load_nb3(I, act && xn < I.nx, xn, y, ym, yp, rym, ryp, z + 1, nb);
            }
            // the adjacent lane's cell next to the pair on plane z
            const R op_ = k ? __shfl_down_sync(0xffffffffu, P0.p0, 1)
                            : __shfl_up_sync(0xffffffffu, P0.p1, 1);
            const R oc_ = k ? __shfl_down_sync(0xffffffffu, P0.c0, 1)
                            : __shfl_up_sync(0xffffffffu, P0.c1, 1);
            const R oa_ = k ? __shfl_down_sync(0xffffffffu, P0.a0, 1)
                            : __shfl_up_sync(0xffffffffu, P0.a1, 1);
            const R ox_ = k ? __shfl_down_sync(0xffffffffu, P0.x0, 1)
                            : __shfl_up_sync(0xffffffffu, P0.x1, 1);
            const int xu = x0 + k;
            if (act && xu < I.nx) {
                const long long c = cell3(I, xu, y, z);
                const R au = k ? P0.a1 : P0.a0, xu_ = k ? P0.x1 : P0.x0;
                const R p0 = k ? P0.p1 : P0.p0, c0 = k ? P0.c1 : P0.c0;
                const R wp = au + I.eps_w, wc = xu_ + I.eps_w;
                R dp = wp, dc = wc, op = cur.rp, oc = cur.rc;
                auto face = [&](R an, R xn, R pn, R cn) {
                    const R fp = hp * (R(0.5) * (wp + (an + I.eps_w)));
                    const R fc = hc * (R(0.5) * (wc + (xn + I.eps_w)));
                    dp += fp;
                    dc += fc;
                    op += fp * pn;
                    oc += fc * cn;
                };
                // the x-neighbour outside the pair: adjacent lane or loaded
                const bool orefl = k ? rxb : rxa;
                R na = oa_, nx_ = ox_, np = op_, nc = oc_;
                if (!orefl && !(k ? shb : sha)) {
                    const long long j = cell3(I, k ? xb : xa, y, z);
                    na = I.a[j];
                    nx_ = I.chi[j];
                    np = I.psi[j];
                    nc = I.C[j];
                }
                // -x, +x: (other, partner) for k = 0, (partner, other) for k = 1
                if (k) {
                    face(P0.a0, P0.x0, P0.p0, P0.c0);
                    if (!orefl) face(na, nx_, np, nc);
                } else {
                    if (!orefl) face(na, nx_, np, nc);
                    if (!rpart) face(P0.a1, P0.x1, P0.p1, P0.c1);
                }
                if (!rym) face(cur.am, cur.xm, cur.pm, cur.cm);
                if (!ryp) face(cur.ap, cur.xp, cur.pp, cur.cp);
                if (!Pm.wall)
                    face(k ? Pm.a1 : Pm.a0, k ? Pm.x1 : Pm.x0, k ? Pm.p1 : Pm.p0,
                         k ? Pm.c1 : Pm.c0);
                if (!Pp.wall)
                    face(k ? Pp.a1 : Pp.a0, k ? Pp.x1 : Pp.x0, k ? Pp.p1 : Pp.p0,
                         k ? Pp.c1 : Pp.c0);
                const R d1 = I.omega * (fdiv(op, dp) - p0), d2 = I.omega * (fdiv(oc, dc) - c0);
                const R p1 = p0 + d1, c1 = c0 + d2;
                I.psi[c] = p1;
                I.C[c] = c1;
                v[0] = fmax(v[0], fabs(d1));
                v[1] = fmax(v[1], fabs(d2));
                v[2] = fmax(v[2], fabs(p1));
                v[3] = fmax(v[3], fabs(c1));
            }
            Pm = P0;
            P0 = Pp;
            Pp = Pn;
        }
    }
    sor3_finish<R, BS>(I, round, colour, v, loop, max_rounds, eager_round);
}

// ---------------------------------------------------------------------------
// k_sor_zm3: one full red-black SOR sweep per launch (Sec. 2.2) with the
// planes of a z-chunk marched through shared memory.  A block owns a TX x TY
// tile of (x, y) and ZC planes of z; it keeps a ring of RING planes of the
// (TX + 4) x (TY + 4) region (the tile and a 2-cell halo): psi, C, the two
// right-hand sides and the weights a, chi.  The planes arrive by
// asynchronous copies (cp.async) issued three steps before their first use,
// so a plane's loads are in flight while the planes before it are swept.  At
// step k the block issues plane k + 4, waits for plane k + 2, updates red on
// plane k + 1 over the tile and a 1-cell ring (the values the neighbouring
// blocks compute for those cells, from the same old black values) and black
// on plane k over the tile, then writes plane k of the tile.  psi and C are
// read from one buffer and written to the other (rounds alternate, as in
// 2D), so no block reads values written in the same launch.  The red phase
// only reads black cells and the black phase only red ones (every periodic
// axis has even length), so the updates are made in place in shared memory.
// The faces are summed in the order of k_sor_rb3, the weights formed as
// there (a + eps_w), so the sweep's values are those of its two half-sweeps.
// ---------------------------------------------------------------------------
template <typename R, int TX, int TY, int ZC, int BS>
struct SorZm {
    static_assert(TX % 2 == 0 && TY % 2 == 0, "z-marching tiles have even sides");
    static constexpr int RX = TX + 4, RY = TY + 4, NP = RX * RY, RING = 6;
    static constexpr int NPT = (NP + BS - 1) / BS;  // region cells a thread copies
    // per ring slot and region cell three pairs: (psi, C), (rhs psi, rhs C),
    // (a, chi); per region cell a flag byte (inside the domain in x and y),
    // per slot one (the plane inside the domain)
    static constexpr size_t smem_bytes() {
        return (size_t)RING * NP * 6 * sizeof(R) + NP + RING + 16;
    }
};

// asynchronous copy of one value from global to shared memory; zero when
// `in` is false (no global read)
template <typename R>
__device__ __forceinline__ void cp_async_val(R *dst, const R *src, bool in) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    if (sizeof(R) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(s), "l"(src),
                     "r"(in ? 4 : 0)
                     : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(s), "l"(src),
                     "r"(in ? 8 : 0)
                     : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;" ::: "memory");
}
// wait until at most N of this thread's most recent groups are pending
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <typename R, int TX, int TY, int ZC, int BS>
__global__ void __launch_bounds__(BS)
    k_sor_zm3(Inst<R> I, cudaGraphConditionalHandle loop, int max_rounds, int eager_round) {
    using T = SorZm<R, TX, TY, ZC, BS>;
    using V = typename Vec2<R>::T;
    constexpr int RX = T::RX, NP = T::NP, RING = T::RING, NPT = T::NPT;
    if (eager_round > 0 && I.ctl->sor_exec < eager_round) return;  // loop already ended
    const int round = I.ctl->sor_exec;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *X = (V *)smem_raw;  // [RING][NP] each
    V *Bv = X + RING * NP, *Wv = Bv + RING * NP;
    uint8_t *flxy = (uint8_t *)(Wv + RING * NP);
    uint8_t *zok = flxy + NP;
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * TX - 2, y0 = blockIdx.y * TY - 2;  // even
    const int zs = blockIdx.z * ZC, ze = min(zs + ZC, I.nz);
    const R *pin = (round & 1) ? I.psi2 : I.psi;
    const R *cin = (round & 1) ? I.C2 : I.C;
    R *pout = (round & 1) ? I.psi : I.psi2;
    R *cout = (round & 1) ? I.C : I.C2;
    const R hp = R(0.5) * I.Ds, hc = R(0.5) * I.Db;
    R v[4] = {R(0), R(0), R(0), R(0)};

    // the region cells this thread copies: their offset in a plane and
    // whether they lie inside the domain in x and y (else they stay zero)
    long long off[NPT];
    bool inxy[NPT];
    int outside = 0;
#pragma unroll
    for (int u = 0; u < NPT; u++) {
        const int q = tid + u * BS;
        off[u] = 0;
        inxy[u] = false;
        if (q < NP) {
            int refl = 0, sx, sy;
            const int Xc = map_axis(x0 + q % RX, I.nx, I.wall[0], 1, refl, sx);
            const int Yc = map_axis(y0 + q / RX, I.ny, I.wall[1], 2, refl, sy);
            inxy[u] = !refl;
            outside |= refl;
            off[u] = (long long)Yc * I.pitch + Xc;
            flxy[q] = (uint8_t)inxy[u];
        }
    }
    // (no region cell beyond a wall or mirror plane in x or y: every face
    // in the plane is taken without reading its flag; block-uniform)
    const bool edge = __syncthreads_or(outside) != 0;
    // issue the copies of plane z (any integer; mapped) into ring slot z mod RING
    auto issue = [&](int z) {
        const int slot = ((z % RING) + RING) % RING;
        int zr = 0, zside;
        const int Z = map_axis(z, I.nz, I.wall[2], 4, zr, zside);
        if (tid == 0) zok[slot] = (uint8_t)!zr;
        const long long base = (long long)Z * I.ny * I.pitch;
#pragma unroll
        for (int u = 0; u < NPT; u++) {
            const int q = tid + u * BS;
            if (q >= NP) continue;
            const bool in = inxy[u] && !zr;
            const long long c = in ? base + off[u] : 0;
            const int k = slot * NP + q;
            cp_async_val((R *)&X[k], pin + c, in);
            cp_async_val((R *)&X[k] + 1, cin + c, in);
            cp_async_val((R *)&Bv[k], I.rpsi + c, in);
            cp_async_val((R *)&Bv[k] + 1, I.rC + c, in);
            cp_async_val((R *)&Wv[k], I.a + c, in);
            cp_async_val((R *)&Wv[k] + 1, I.chi + c, in);
        }
    };
    // one cell update at region index q of ring slot s0 (neighbour planes in
    // slots sm, spl, inside the domain when zm, zp); the six faces in the
    // order -x, +x, -y, +y, plane below, plane above; no flux across a wall
    // or out of the domain
    auto update = [&](int s0, int sm, int spl, bool zm, bool zp, int q, bool track) {
        const int k = s0 * NP + q;
        const V w0 = Wv[k], b0 = Bv[k];
        const R w0p = w0.x + I.eps_w, w0c = w0.y + I.eps_w;
        R dp = w0p, dc = w0c, op = b0.x, oc = b0.y;
        const int nbk[6] = {k - 1, k + 1, k - RX, k + RX, sm * NP + q, spl * NP + q};
        bool nin[6] = {true, true, true, true, zm, zp};
        if (edge) {
            nin[0] = flxy[q - 1] != 0;
            nin[1] = flxy[q + 1] != 0;
            nin[2] = flxy[q - RX] != 0;
            nin[3] = flxy[q + RX] != 0;
        }
#pragma unroll
        for (int f = 0; f < 6; f++) {
            if (!nin[f]) continue;
            const int j = nbk[f];
            const V wj = Wv[j], xj = X[j];
            const R fp = hp * (R(0.5) * (w0p + (wj.x + I.eps_w)));
            const R fc = hc * (R(0.5) * (w0c + (wj.y + I.eps_w)));
            dp += fp;
            dc += fc;
            op += fp * xj.x;
            oc += fc * xj.y;
        }
        const V x0v = X[k];
        const R d1 = I.omega * (fdiv(op, dp) - x0v.x), d2 = I.omega * (fdiv(oc, dc) - x0v.y);
        const R p1 = x0v.x + d1, c1 = x0v.y + d2;
        X[k] = V{p1, c1};
        if (track) {
            v[0] = fmax(v[0], fabs(d1));
            v[1] = fmax(v[1], fabs(d2));
            v[2] = fmax(v[2], fabs(p1));
            v[3] = fmax(v[3], fabs(c1));
        }
    };
    const bool zwall = I.wall[2] != 0;
    // step k needs planes k - 1 .. k + 2 (red of k + 1, black of k).  The
    // march starts at k = zs - 2 (red of the plane below the chunk); planes
    // zs - 2 .. zs + 1 go out first, and step k issues plane k + 4 into the
    // slot of plane k - 2 (last read by the black phase of step k - 1).
    for (int z = zs - 2; z <= zs + 1; z++) {
        issue(z);
        cp_async_commit();
    }
    for (int k = zs - 2; k < ze; k++) {
        if (k + 4 <= ze + 1) issue(k + 4);
        cp_async_commit();  // (an empty group past the chunk keeps the count)
        cp_async_wait<2>();  // this thread's copies of planes <= k + 2 landed
        __syncthreads();
        // red on plane k + 1 over the tile and a 1-cell ring: thread t takes
        // red cell t of the (TX + 2) x (TY + 2) ring region, row by row
        // (red: x + y + z even; a periodic wrap of even length keeps the
        // parity, a reflected cell is outside)
        if (k + 1 <= ze) {
            const int zr = k + 1;
            const bool zin = zr >= 0 && zr < I.nz;
            const int s0 = ((zr % RING) + RING) % RING;
            if ((zin || !zwall) && zok[s0]) {
                const int sm = (s0 + RING - 1) % RING, spl = (s0 + 1) % RING;
                const bool zm = zok[sm] != 0, zp = zok[spl] != 0;
                constexpr int HX = (TX + 2) / 2, NRED = HX * (TY + 2);
                for (int t = tid; t < NRED; t += BS) {
                    const int ry = 1 + t / HX, j = t - (ry - 1) * HX;
                    const int p = (x0 + y0 + ry + zr) & 1;
                    const int rx = 2 - p + 2 * j;
                    const int q = ry * RX + rx;
                    if (edge && !flxy[q]) continue;
                    const int gx = x0 + rx, gy = y0 + ry;
                    const bool own = rx >= 2 && rx < 2 + TX && ry >= 2 && ry < 2 + TY &&
                                     gx < I.nx && gy < I.ny && zr >= zs && zr < ze;
                    update(s0, sm, spl, zm, zp, q, own);
                }
            }
        }
        __syncthreads();
        // black on plane k over the tile: thread t takes black cell t
        if (k >= zs) {
            const int s0 = ((k % RING) + RING) % RING;
            const int sm = (s0 + RING - 1) % RING, spl = (s0 + 1) % RING;
            const bool zm = zok[sm] != 0, zp = zok[spl] != 0;
            constexpr int HX = TX / 2, NBL = HX * TY;
            for (int t = tid; t < NBL; t += BS) {
                const int ry = 2 + t / HX, j = t - (ry - 2) * HX;
                const int p = (x0 + y0 + ry + k) & 1;
                const int rx = 3 - p + 2 * j;  // black: x + y + z odd
                const int gx = x0 + rx, gy = y0 + ry;
                if (gx >= I.nx || gy >= I.ny) continue;
                update(s0, sm, spl, zm, zp, ry * RX + rx, true);
            }
        }
        __syncthreads();
        // write plane k of the tile
        if (k >= zs) {
            const int s0 = ((k % RING) + RING) % RING;
            for (int a = tid; a < TX * TY; a += BS) {
                const int rx = 2 + a % TX, ry = 2 + a / TX;
                const int gx = x0 + rx, gy = y0 + ry;
                if (gx >= I.nx || gy >= I.ny) continue;
                const long long c = ((long long)k * I.ny + gy) * I.pitch + gx;
                const V xs = X[s0 * NP + ry * RX + rx];
                pout[c] = xs.x;
                cout[c] = xs.y;
            }
        }
    }
    cp_async_wait<0>();
    __syncthreads();
    // block maxima of the sweep -> round slot; the last block decides
    __shared__ R sh[4][BS / 32];
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
    const unsigned int nb = gridDim.x * gridDim.y * gridDim.z;
    if (!last_block(&I.ctl->sor_ticket, nb)) return;
    if (tid != 0) return;
    Ctl *ctl = I.ctl;
    ctl->sor_ticket = 0;
    const bool stop = sor_round_stop<R>(ctl, round, double(I.sor_tol), max_rounds);
    if (eager_round < 0) {
        ctl->sor_exec = round + 1;
        if (stop) cudaGraphSetConditional(loop, 0);
    } else {
        ctl->sor_exec = stop ? -(round + 1) - 1000000 : round + 1;
    }
}

#undef LBS_CELL3

}  // namespace lbs
