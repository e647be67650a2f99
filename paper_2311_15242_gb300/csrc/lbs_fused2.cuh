// lbs_fused2.cuh — the D2Q9 coupled step as two launches (arXiv 2311.15242,
// Secs. 2.1-2.2).
//
//   k_lbfd2     one pass over a TX x TY tile of cells with a 3-cell halo in
//               shared memory: normals, curvature, interfacial force and
//               velocity (Eqs. 5-10), the explicit surfactant terms and the
//               Crank-Nicolson right-hand sides (Eqs. 22-28), collision and
//               recolouring (Eqs. 1-4, 11-12, App. A) of the tile and of the
//               ring of cells around it, and streaming in pull form
//               (Eq. 13) from the collided ring and tile in shared memory.
//               Post-collision populations never reach global memory.
//   k_sorfuse2  one cooperative launch: colour gradient and weights at t+1,
//               every round of the blocked red-black SOR (Sec. 2.2), the
//               conserved total and the rescale, with grid barriers between
//               the phases.
//
// Populations ping-pong between the two sets of the workspace by the parity
// of the step counter: the state at step s lives in set s & 1 (pull form
// reads neighbours' values, so a step cannot write the set it reads).  So do
// the moments rho^R, rho^B, rho^N, j (mom_set): k_lbfd2 reads those of t and
// writes those of t+1 to the other set, which the SOR launch's first phase
// reads for the gradient of t+1.
#pragma once

#include "lbs_k2d.cuh"

namespace lbs {

// code of a halo slot: bit 0 / 1 the slot lies beyond the wall or mirror
// plane of axis x / y and holds the mirror image of its source cell; bit 2 / 3
// that boundary is the high end of the axis; bit 4 the slot has no source
// cell (more than one reflection away: never read)
enum : uint8_t { RC_RX = 1, RC_RY = 2, RC_HX = 4, RC_HY = 8, RC_NONE = 16 };

template <typename R, int TX, int TY>
struct Fuse2 {
    static constexpr int W3 = TX + 6, H3 = TY + 6, N3 = W3 * H3;  // halo 3
    static constexpr int W2 = TX + 4, H2 = TY + 4, N2 = W2 * H2;  // halo 2
    static constexpr int W1 = TX + 2, H1 = TY + 2, N1 = W1 * H1;  // halo 1
    static constexpr int NT = TX * TY;                            // threads
    static constexpr int NRING = 2 * (TX + 2) + 2 * TY;
    static_assert(NRING <= NT, "the ring of a tile is collided by one pass of its threads");
    // R planes: g (2), psi, n (2) over halo 3; rho^R, rho^B, j (2), a, chi,
    // C, u (2), F (2) over halo 2; post-collision moving populations (8 + 8)
    // and rest populations (2) over halo 1
    static constexpr size_t r_count = 5 * (size_t)N3 + 11 * (size_t)N2 + 18 * (size_t)N1;
    static constexpr size_t bytes() {
        return r_count * sizeof(R) + N3 + N1 + 2 * (size_t)N1 + 16;
    }
    __device__ static constexpr int i3(int x, int y) { return (y + 3) * W3 + x + 3; }
    __device__ static constexpr int i2(int x, int y) { return (y + 2) * W2 + x + 2; }
    __device__ static constexpr int i1(int x, int y) { return (y + 1) * W1 + x + 1; }
};

// the value stq would store and return, without storing it
template <typename R, typename P>
__device__ __forceinline__ R round_pop(const Inst<R> &I, R v, unsigned int r) {
    const P s = PopCvt<P>::from_r(PopCvt<P>::scaled ? v * I.pscale : v, r);
    const R back = R(PopCvt<P>::to(s));
    return PopCvt<P>::scaled ? back * I.pinv : back;
}

// the population sets of the current step (src) and of the next (dst), and
// the moment planes of both
template <typename R>
struct PopSets {
    const void *sT, *sM;
    const R *sT0, *sM0;
    const uint8_t *sflag;
    void *dT, *dM;
    R *dT0, *dM0;
    uint8_t *dflag;
    MomSet<R> sm, dm;
};
template <typename R>
__device__ __forceinline__ PopSets<R> pop_sets(const Inst<R> &I) {
    const bool odd = I.pop_pp && (I.ctl->step & 1);
    PopSets<R> p;
    p.sT = odd ? I.gT : I.fT;
    p.sM = odd ? I.gM : I.fM;
    p.sT0 = odd ? I.gT0 : I.fT0;
    p.sM0 = odd ? I.gM0 : I.fM0;
    p.sflag = odd ? I.gflag : I.flag;
    p.dT = odd ? I.fT : I.gT;
    p.dM = odd ? I.fM : I.gM;
    p.dT0 = odd ? I.fT0 : I.gT0;
    p.dM0 = odd ? I.fM0 : I.gM0;
    p.dflag = odd ? I.flag : I.gflag;
    p.sm = mom_set(I, odd);
    p.dm = mom_set(I, !odd);
    return p;
}

// phases 2-6 of k_lbfd2 over the loaded tile; EDGE (block-uniform): the
// tile's halo holds mirror images (walls, mirror planes), so the reflection
// codes are read; without it every slot is a cell of the grid and every link
// a plain pull.  It is tested at run time, not compiled into two versions:
// the cells a tile recomputes from its neighbours' data (forces in the halo,
// collisions of the ring) must come out bit for bit as the neighbour's own,
// since the owner closes each cell's mass with the populations it streams
// out, and a differently compiled copy could fuse other multiply-adds.
template <typename R, typename P, int TX, int TY>
__device__ __forceinline__ void lbfd2_tile(const Inst<R> &I, const PopSets<R> &ps,
                                           unsigned char *smem_raw, const bool EDGE) {
    using F = Fuse2<R, TX, TY>;
    constexpr int W3 = F::W3, N3 = F::N3, W2 = F::W2, N2 = F::N2, W1 = F::W1, N1 = F::N1;
    constexpr int NT = F::NT;
    R *gx3 = (R *)smem_raw, *gy3 = gx3 + N3, *ps3 = gy3 + N3, *nx3 = ps3 + N3, *ny3 = nx3 + N3;
    R *rR2 = ny3 + N3, *rB2 = rR2 + N2, *jx2 = rB2 + N2, *jy2 = jx2 + N2, *a2 = jy2 + N2;
    R *ch2 = a2 + N2, *Cs2 = ch2 + N2, *ux2 = Cs2 + N2, *uy2 = ux2 + N2, *Fx2 = uy2 + N2;
    R *Fy2 = Fx2 + N2;
    R *pT1 = Fy2 + N2, *pM1 = pT1 + 8 * N1, *pT01 = pM1 + 8 * N1, *pM01 = pT01 + N1;
    uint8_t *code3 = (uint8_t *)(pM01 + N1), *flag1 = code3 + N3;
    int16_t *src1 = (int16_t *)(((uintptr_t)(flag1 + N1) + 1) & ~(uintptr_t)1);
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;

    // 2. interface normals n = -g / sqrt(|g|^2 + eps_n^2) (reading R3)
    const R e2 = I.eps_n * I.eps_n;
    for (int q = tid; q < N3; q += NT) {
        const R inv = frsq(gx3[q] * gx3[q] + gy3[q] * gy3[q] + e2);
        nx3[q] = -gx3[q] * inv;
        ny3[q] = -gy3[q] * inv;
    }
    __syncthreads();

    // 3. force and velocity (Eqs. 5-10, buoyancy of Sec. 3.4) at every cell of
    //    the halo-2 region that is a cell of the grid (not a mirror image)
    for (int q = tid; q < N2; q += NT) {
        const int x = q % W2 - 2, y = q / W2 - 2;
        const int k3 = F::i3(x, y);
        if (EDGE && (code3[k3] & (RC_RX | RC_RY | RC_NONE))) continue;
        R divn = R(0), dpx = R(0), dpy = R(0);
#pragma unroll
        for (int i = 1; i < Q9; i++) {
            const int j = k3 + ex9(i) + ey9(i) * W3;
            divn += w9<R>(i) * (R(ex9(i)) * nx3[j] + R(ey9(i)) * ny3[j]);
            const R p = ps3[j];
            dpx += w9<R>(i) * R(ex9(i)) * p;
            dpy += w9<R>(i) * R(ey9(i)) * p;
        }
        const R kappa = -R(3) * divn;
        dpx *= R(3);
        dpy *= R(3);
        const R gx = gx3[k3], gy = gy3[k3], a = a2[q];
        R sigma, mco, Fx, Fy;
        if (eos(I, ps3[k3], sigma, mco)) {
            const R nx = nx3[k3], ny = ny3[k3];
            const R ndp = nx * dpx + ny * dpy;
            Fx = -R(0.5) * sigma * kappa * gx - R(0.5) * a * mco * (dpx - ndp * nx);
            Fy = -R(0.5) * sigma * kappa * gy - R(0.5) * a * mco * (dpy - ndp * ny);
        } else {
            Fx = -R(0.5) * I.sigma_min * kappa * gx;
            Fy = -R(0.5) * I.sigma_min * kappa * gy;
        }
        const R rR = rR2[q], rB = rB2[q];
        const R rho = rR + rB;
        const R drb = rR + (rB - I.rhoB0);
        Fx += drb * I.g[0];
        Fy += drb * I.g[1];
        Fx2[q] = Fx;
        Fy2[q] = Fy;
        const R irho = fdiv(R(1), rho);
        ux2[q] = (jx2[q] + R(0.5) * Fx) * irho;
        uy2[q] = (jy2[q] + R(0.5) * Fy) * irho;
    }
    __syncthreads();
    // mirror images: the velocity and force of the source cell with the
    // normal components mirrored (the source is a cell of this tile)
    if (EDGE) {
    for (int q = tid; q < N2; q += NT) {
        const int x = q % W2 - 2, y = q / W2 - 2;
        const uint8_t cd = code3[F::i3(x, y)];
        if (!(cd & (RC_RX | RC_RY)) || (cd & RC_NONE)) continue;
        int refl = 0, sx, sy;
        const int sxt = (cd & RC_RX) ? map_axis(x0 + x, I.nx, I.wall[0], 1, refl, sx) - x0 : x;
        const int syt = (cd & RC_RY) ? map_axis(y0 + y, I.ny, I.wall[1], 2, refl, sy) - y0 : y;
        // (images more than two cells beyond the boundary are never read)
        if (sxt < -2 || sxt >= TX + 2 || syt < -2 || syt >= TY + 2) continue;
        const int s = F::i2(sxt, syt);
        R u0 = ux2[s], u1 = uy2[s], f0 = Fx2[s], f1 = Fy2[s];
        if (cd & RC_RX) {
            u0 = -u0;
            f0 = -f0;
        }
        if (cd & RC_RY) {
            u1 = -u1;
            f1 = -f1;
        }
        ux2[q] = u0;
        uy2[q] = u1;
        Fx2[q] = f0;
        Fy2[q] = f1;
    }
    __syncthreads();
    }

    // 4. the explicit surfactant terms and right-hand sides of the tile's
    //    cells (Eqs. 22-28), and the SOR starting guess 2 x^t - x^(t-1)
    const int tx = tid % TX, ty = tid / TX;
    const bool own = x0 + tx < I.nx && y0 + ty < I.ny;
    const long long c = (long long)(y0 + ty) * I.pitch + (x0 + tx);
    if (own && I.transport) {
        R Px[5], Cx[5], Py[5], Cy[5];
#pragma unroll
        for (int k = -2; k <= 2; k++) {
            int j3 = F::i3(tx + k, ty), j2 = F::i2(tx + k, ty);
            uint8_t cd = EDGE ? code3[j3] : 0;
            R sgn = (cd & RC_RX) ? R(-1) : R(1);
            R u = (cd & RC_RX) ? -ux2[j2] : ux2[j2];  // the source cell's own value
            Px[k + 2] = sgn * ps3[j3] * a2[j2] * u;
            Cx[k + 2] = sgn * Cs2[j2] * ch2[j2] * u;
            j3 = F::i3(tx, ty + k);
            j2 = F::i2(tx, ty + k);
            cd = EDGE ? code3[j3] : 0;
            sgn = (cd & RC_RY) ? R(-1) : R(1);
            u = (cd & RC_RY) ? -uy2[j2] : uy2[j2];
            Py[k + 2] = sgn * ps3[j3] * a2[j2] * u;
            Cy[k + 2] = sgn * Cs2[j2] * ch2[j2] * u;
        }
        const int k2 = F::i2(tx, ty), k3 = F::i3(tx, ty);
        const R ux = ux2[k2], uy = uy2[k2];
        const R divP = upwind(Px + 2, ux) + upwind(Py + 2, uy);
        const R divC = upwind(Cx + 2, ux) + upwind(Cy + 2, uy);
        const R psi = ps3[k3], Cc = Cs2[k2], a = a2[k2];
        const R j = I.source == 1 ? I.ra * I.psi_inf * Cc
                                  : I.ra * Cc * (I.psi_inf - psi) - I.rd * psi;
        const R S = -divP + a * j;
        const R B = -divC - a * j;
        const R wp = a + I.eps_w, wc = ch2[k2] + I.eps_w;
        R Lp = R(0), Lc = R(0);
#pragma unroll
        for (int f = 0; f < 4; f++) {
            const int dx = f == 0 ? -1 : (f == 1 ? 1 : 0);
            const int dy = f == 2 ? -1 : (f == 3 ? 1 : 0);
            const int j3 = F::i3(tx + dx, ty + dy), j2 = F::i2(tx + dx, ty + dy);
            if (EDGE && (code3[j3] & (RC_RX | RC_RY))) continue;  // no flux through a wall
            Lp += R(0.5) * (wp + (a2[j2] + I.eps_w)) * (ps3[j3] - psi);
            Lc += R(0.5) * (wc + (ch2[j2] + I.eps_w)) * (Cs2[j2] - Cc);
        }
        const bool first = I.ctl->step == 0;
        const R Sp = I.S[c], Bp = I.B[c];
        const R abS = first ? S : R(1.5) * S - R(0.5) * Sp;
        const R abB = first ? B : R(1.5) * B - R(0.5) * Bp;
        I.rpsi[c] = wp * psi + R(0.5) * I.Ds * Lp + abS;
        I.rC[c] = wc * Cc + R(0.5) * I.Db * Lc + abB;
        I.S[c] = S;
        I.B[c] = B;
        // starting guess of the solve in the second buffers (round 0 reads
        // them); this time level becomes the previous one
        I.psi2[c] = R(2) * psi - I.psip[c];
        I.C2[c] = R(2) * Cc - I.Cp[c];
        I.psip[c] = psi;
        I.Cp[c] = Cc;
    }

    // 5. collision and recolouring (Eqs. 1-4, 11-12) of the tile's cells
    //    (pass 0) and of the ring around it (pass 1), into shared memory.
    //    A ring slot beyond a mirror plane points at its source cell's slot;
    //    one beyond a bounce-back wall is never read.
#pragma unroll 1
    for (int pass = 0; pass < 2; pass++) {
        int x, y;
        if (pass == 0) {
            x = tx;
            y = ty;
        } else {
            if (tid >= F::NRING) break;
            const int r = tid;
            if (r < TX + 2) {
                x = r - 1;
                y = -1;
            } else if (r < 2 * (TX + 2)) {
                x = r - (TX + 2) - 1;
                y = TY;
            } else if (r < 2 * (TX + 2) + TY) {
                x = -1;
                y = r - 2 * (TX + 2);
            } else {
                x = TX;
                y = r - 2 * (TX + 2) - TY;
            }
        }
        const int p1 = F::i1(x, y), k3 = F::i3(x, y), k2 = F::i2(x, y);
        const uint8_t cd = EDGE ? code3[k3] : 0;
        if (cd & RC_NONE) {
            src1[p1] = -1;
            continue;
        }
        if (cd & (RC_RX | RC_RY)) {
            const int r = cd & (RC_RX | RC_RY);
            if (r & I.bbmask) {
                src1[p1] = -1;
                continue;
            }
            int refl = 0, sx, sy;
            const int sxt = (cd & RC_RX) ? map_axis(x0 + x, I.nx, I.wall[0], 1, refl, sx) - x0 : x;
            const int syt = (cd & RC_RY) ? map_axis(y0 + y, I.ny, I.wall[1], 2, refl, sy) - y0 : y;
            const bool in1 = sxt >= -1 && sxt < TX + 1 && syt >= -1 && syt < TY + 1;
            src1[p1] = in1 ? (int16_t)F::i1(sxt, syt) : (int16_t)-1;
            continue;
        }
        src1[p1] = (int16_t)p1;
        int refl = 0, sxx, syy;
        const int X = map_axis(x0 + x, I.nx, I.wall[0], 1, refl, sxx);
        const int Y = map_axis(y0 + y, I.ny, I.wall[1], 2, refl, syy);
        const long long cc = (long long)Y * I.pitch + X;
        (void)refl;
        R fT[Q9], fM[Q9];
        const int fl = ps.sflag[cc];
        fT[0] = ps.sT0[cc];
        fM[0] = ps.sM0[cc];
#pragma unroll
        for (int i = 1; i < Q9; i++) {
            fT[i] = ldp<R, P>(I, ps.sT, (long long)i * I.plane + cc);
            fM[i] = ldp<R, P>(I, ps.sM, (long long)i * I.plane + cc);
        }
        Mom2<R> mo = moments9(I, fT, fM, fl);
        const R rR = mo.rR, rB = mo.rB;
        const R rmin = fl ? rB : rR;
        const R devmaj = I.dsh[fl] + (mo.drho - rmin);
        const R rho = rR + rB;
        const R ux = ux2[k2], uy = uy2[k2], Fx = Fx2[k2], Fy = Fy2[k2];
        // d_a(rho^k u_a), u at walls as the ghost velocity
        R dRx = R(0), dRy = R(0), dBx = R(0), dBy = R(0);
#pragma unroll
        for (int i = 1; i < Q9; i++) {
            const int j2 = k2 + ex9(i) + ey9(i) * W2;
            R vx = ux2[j2], vy = uy2[j2];
            if (EDGE) {
                const uint8_t cj = code3[k3 + ex9(i) + ey9(i) * W3];
                const int rj = cj & (RC_RX | RC_RY);
                if (rj & 1) vx = -vx;  // back to the source cell's own velocity
                if (rj & 2) vy = -vy;
                const int sx = (rj & 1) ? ((cj & RC_HX) ? 1 : -1) : 0;
                const int sy = (rj & 2) ? ((cj & RC_HY) ? 1 : -1) : 0;
                ghost_u2(I, rj, sx, sy, vx, vy);
            }
            const R r1 = rR2[j2], r2 = rB2[j2];
            const R wx = w9<R>(i) * R(ex9(i)), wy = w9<R>(i) * R(ey9(i));
            dRx += wx * r1 * vx;
            dRy += wy * r1 * vy;
            dBx += wx * r2 * vx;
            dBy += wy * r2 * vy;
        }
        const R cR = R(1.8) * I.alphaR - R(0.8), cB = R(1.8) * I.alphaB - R(0.8);
        const R Qx = R(3) * (cR * dRx + cB * dBx), Qy = R(3) * (cR * dRy + cB * dBy);
        // the non-conserved moments of Eq. 36 (rows e, epsilon, q_x, q_y,
        // p_xx, p_xy) of the shifted totals, from partial sums of the axis
        // (1-4) and diagonal (5-8) directions
        R mT[Q9];
        {
            const R a13 = fT[1] + fT[3], a24 = fT[2] + fT[4];
            const R a57 = fT[5] + fT[7], a68 = fT[6] + fT[8];
            const R S1 = a13 + a24, S2 = a57 + a68;
            const R d13 = fT[1] - fT[3], d24 = fT[2] - fT[4];
            const R d57 = fT[5] - fT[7], d86 = fT[8] - fT[6];
            mT[0] = mT[3] = mT[5] = R(0);  // (not used: conserved rows)
            mT[1] = (R(2) * S2 - S1) - R(4) * fT[0];
            mT[2] = (S2 - R(2) * S1) + R(4) * fT[0];
            mT[4] = (d57 + d86) - R(2) * d13;
            mT[6] = (d57 - d86) - R(2) * d24;
            mT[7] = a13 - a24;
            mT[8] = a57 - a68;
        }
        const R u2 = ux * ux + uy * uy;
        const R aBm = R(3.6) * I.alphaB + R(0.4), aRm = R(3.6) * I.alphaR + R(0.4);
        const R bBm = R(5.4) * I.alphaB - R(1.4), bRm = R(5.4) * I.alphaR - R(1.4);
        const R qco = R(-1.8) * (I.alphaR * rR + I.alphaB * rB) - R(0.2) * rho;
        R neq[Q9];
        neq[0] = R(0);
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
        const R rN = colour_fn(I, rR, rB);
        const R inv_mu = (R(1) + rN) * I.inv_2muR + (R(1) - rN) * I.inv_2muB;
        const R pk = rR * I.cs2R + rB * I.cs2B;
        const R sv = fdiv(R(1), R(0.5) + fdiv(R(1), inv_mu * pk));
        const R Sd[Q9] = {R(0), R(1.25), R(1.14), R(0), R(1.6), R(0), R(1.6), sv, sv};
        const R uF = ux * Fx + uy * Fy;
        const R Fh[Q9] = {R(0), R(6) * uF, R(-6) * uF, Fx, -Fx, Fy, -Fy,
                          R(2) * (ux * Fx - uy * Fy), ux * Fy + uy * Fx};
        const R Cm[Q9] = {R(0), R(3) * (Qx + Qy), R(0), R(0), R(0), R(0), R(0), Qx - Qy, R(0)};
        R dm[Q9];
#pragma unroll
        for (int jm = 0; jm < Q9; jm++)
            dm[jm] = (-Sd[jm] * neq[jm] + (R(1) - R(0.5) * Sd[jm]) * (Cm[jm] + Fh[jm])) *
                     (R(1) / R(mnorm9(jm)));
        // f + M^T dm (dm already divided by the row norms; dm_0 = 0): the
        // columns of Eq. 36 share the axis and diagonal combinations
        R post[Q9];
        {
            const R A = -dm[1] - R(2) * dm[2], Bd = R(2) * dm[1] + dm[2];
            const R X1 = dm[3] - R(2) * dm[4], Y1 = dm[5] - R(2) * dm[6];
            const R X2 = dm[3] + dm[4], Y2 = dm[5] + dm[6];
            post[0] = fT[0] + (R(4) * dm[2] - R(4) * dm[1]);
            post[1] = fT[1] + ((A + X1) + dm[7]);
            post[2] = fT[2] + ((A + Y1) - dm[7]);
            post[3] = fT[3] + ((A - X1) + dm[7]);
            post[4] = fT[4] + ((A - Y1) - dm[7]);
            post[5] = fT[5] + ((Bd + X2) + (Y2 + dm[8]));
            post[6] = fT[6] + ((Bd - X2) + (Y2 - dm[8]));
            post[7] = fT[7] + ((Bd - X2) - (Y2 - dm[8]));
            post[8] = fT[8] + ((Bd + X2) - (Y2 + dm[8]));
        }
        CSum<R> rdc;
#pragma unroll
        for (int i = 0; i < Q9; i++) rdc.add(shift_of(I, i, fl) + post[i]);
        const R rdag = rdc.value();
        const R ggx = gx3[k3], ggy = gy3[k3];
        const R seg = I.beta * rR * rB * R(3) * pk *
                      frsq(ggx * ggx + ggy * ggy + I.eps_n * I.eps_n) * fdiv(R(1), rho * rho);
        const R fr = fdiv(rmin, rdag);
        const R sg = fl ? R(-1) : R(1);
        CSum<R> sT, sM;
        const unsigned int rk = rest_key(cc, rest_salt(0, I.ctl->step)), rs = pop_seed(rk);
#pragma unroll
        for (int i = 1; i < Q9; i++) {
            const R segi = seg * w9<R>(i) * (R(ex9(i)) * ggx + R(ey9(i)) * ggy);
            const R vT = round_pop<R, P>(I, post[i], pop_r(rs, 2 * i));
            const R vM = round_pop<R, P>(I, fr * (I.shift[i] + post[i]) + sg * segi,
                                         pop_r(rs, 2 * i + 1));
            pT1[(i - 1) * N1 + p1] = vT;
            pM1[(i - 1) * N1 + p1] = vM;
            sT.add(vT);
            sM.add(vM);
        }
        pT01[p1] = rest_close(mo.dr_s, mo.dr_c, sT.s, sT.c, R(0), rest_u(rk, 0));
        pM01[p1] = rest_close(mo.rm_s, mo.rm_c, sM.s, sM.c, R(0), rest_u(rk, 1));
        flag1[p1] = (uint8_t)fl;
    }
    __syncthreads();

    // 6. streaming into the tile's cells (pull form, Eq. 13): a link across a
    //    bounce-back wall returns the cell's own opposite population (a
    //    moving wall adds 2 w_i rho^k (e_i . u_w) / c_s^2); across mirror
    //    planes it brings the mirrored population of the mirrored cell.
    //    The moments of t+1 go to the next-moment planes.
    if (!own) return;
    const int p1 = F::i1(tx, ty), k3c = F::i3(tx, ty), k2c = F::i2(tx, ty);
    const int flc = flag1[p1];
    R t[Q9], m[Q9];
    unsigned slow = 0, fbits = 0;
    t[0] = pT01[p1];
    m[0] = pM01[p1];
#pragma unroll
    for (int i = 1; i < Q9; i++) {
        const uint8_t cj = EDGE ? code3[k3c - ex9(i) - ey9(i) * W3] : 0;
        const int refl = cj & (RC_RX | RC_RY);
        const int bb = refl & I.bbmask;
        const int src = EDGE ? (bb ? p1 : src1[p1 - ex9(i) - ey9(i) * W1])
                             : p1 - ex9(i) - ey9(i) * W1;
        const int k = EDGE ? (bb ? opp9(i) : mir9(i, refl)) : i;
        t[i] = pT1[(k - 1) * N1 + src];
        m[i] = pM1[(k - 1) * N1 + src];
        const int fj = flag1[src];
        fbits |= (unsigned)fj << i;
        if (fj != flc || (bb & I.mvmask)) slow |= 1u << i;
    }
    fbits |= (unsigned)flc;
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
                stp<R, P>(I, ps.dT, (long long)i * I.plane + c, t[i]);
                stp<R, P>(I, ps.dM, (long long)i * I.plane + c, m[i]);
            }
            ps.dT0[c] = t[0];
            ps.dM0[c] = m[0];
            ps.dflag[c] = (uint8_t)flc;
            ps.dm.rR[c] = rR;
            ps.dm.rB[c] = rB;
            ps.dm.rN[c] = colour_fn(I, rR, rB);
            ps.dm.jx[c] = jx;
            ps.dm.jy[c] = jy;
            return;
        }
    }
    const R rRc = rR2[k2c], rBc = rB2[k2c];
    R fR[Q9], fB[Q9];
    R loT = R(0), loR = R(0), loB = R(0);
#pragma unroll
    for (int i = 0; i < Q9; i++) {
        const int fj = (fbits >> i) & 1;
        R tlo = R(0), mlo = R(0);
        R sh = shift_of(I, i, fj);
        if ((slow >> i) & 1) {
            const uint8_t cj = code3[k3c - ex9(i) - ey9(i) * W3];
            const int refl = cj & (RC_RX | RC_RY) & I.bbmask;
            if (refl) {
                R uwx = R(0), uwy = R(0);
                int nw = 0;
                if (refl & 1) {
                    const R *w = (cj & RC_HX) ? I.uw_hi[0] : I.uw_lo[0];
                    uwx += w[0];
                    uwy += w[1];
                    nw++;
                }
                if (refl & 2) {
                    const R *w = (cj & RC_HY) ? I.uw_hi[1] : I.uw_lo[1];
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
    if (fl != flc) {
        R d1, d2;
        const R d = two_sum(I.shift0[flc], -I.shift0[fl], d1);
        t[0] = two_sum(d, t[0], d2);
        loT += d1 + d2;
    }
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
            fT[i] = stq_r<R, P>(I, ps.dT, i, c, t[i], pop_r(rs, 2 * i));
            fM[i] = stq_r<R, P>(I, ps.dM, i, c, mh, pop_r(rs, 2 * i + 1));
            sT.add(fT[i]);
            sM.add(fM[i]);
        }
    }
    fT[0] = rest_close(gT.s, gT.c, sT.s, sT.c, loT, rest_u(rk, 0));
    fM[0] = rest_close(gM.s, gM.c, sM.s, sM.c, loM, rest_u(rk, 1));
    ps.dT0[c] = fT[0];
    ps.dM0[c] = fM[0];
    ps.dflag[c] = (uint8_t)fl;
    const Mom2<R> mo = moments9(I, fT, fM, fl);
    ps.dm.rR[c] = mo.rR;
    ps.dm.rB[c] = mo.rB;
    ps.dm.rN[c] = colour_fn(I, mo.rR, mo.rB);
    ps.dm.jx[c] = mo.jx;
    ps.dm.jy[c] = mo.jy;
}

template <typename R, typename P, int TX, int TY>
__global__ void __launch_bounds__(TX * TY, (sizeof(R) == 4 ? 1024 : 512) / (TX * TY)) k_lbfd2(Inst<R> I) {
    using F = Fuse2<R, TX, TY>;
    constexpr int W3 = F::W3, N3 = F::N3, N2 = F::N2, N1 = F::N1;
    constexpr int NT = F::NT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // the halo slots this phase fills (layout as in lbfd2_tile)
    R *gx3 = (R *)smem_raw, *gy3 = gx3 + N3, *ps3 = gy3 + N3;
    R *rR2 = ps3 + 3 * N3, *rB2 = rR2 + N2, *jx2 = rB2 + N2, *jy2 = jx2 + N2, *a2 = jy2 + N2;
    R *ch2 = a2 + N2, *Cs2 = ch2 + N2;
    uint8_t *code3 = (uint8_t *)(rR2 + 11 * N2 + 18 * N1);
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const PopSets<R> ps = pop_sets(I);
    // the one-launch SOR follows: its grid barrier starts from a clear count
    // whatever an earlier launch that gave up left behind
    if (blockIdx.x == 0 && blockIdx.y == 0 && tid == 0) I.ctl->bar_count = 0;

    // 1. the halo-3 region: g (normal component mirrored at walls and
    //    mirror planes), psi; the halo-2 part also rho^R, rho^B, j, a, chi, C
    int near_edge = 0;  // a slot of this thread is a mirror image or has no source
    for (int q = tid; q < N3; q += NT) {
        const int x = q % W3 - 3, y = q / W3 - 3;
        int refl = 0, sx, sy;
        const int X = map_axis(x0 + x, I.nx, I.wall[0], 1, refl, sx);
        const int Y = map_axis(y0 + y, I.ny, I.wall[1], 2, refl, sy);
        const bool valid = X >= 0 && X < I.nx && Y >= 0 && Y < I.ny;
        code3[q] = (uint8_t)((refl & 3) | (sx > 0 ? RC_HX : 0) | (sy > 0 ? RC_HY : 0) |
                             (valid ? 0 : RC_NONE));
        near_edge |= (refl & 3) | !valid;
        const bool h2 = x >= -2 && x < TX + 2 && y >= -2 && y < TY + 2;
        const int k = F::i2(x, y);
        if (valid) {
            const long long c = (long long)Y * I.pitch + X;
            R g0 = I.gx[c], g1 = I.gy[c];
            if (refl & 1) g0 = -g0;
            if (refl & 2) g1 = -g1;
            gx3[q] = g0;
            gy3[q] = g1;
            ps3[q] = I.psi[c];
            if (h2) {
                rR2[k] = ps.sm.rR[c];
                rB2[k] = ps.sm.rB[c];
                jx2[k] = ps.sm.jx[c];
                jy2[k] = ps.sm.jy[c];
                a2[k] = I.a[c];
                ch2[k] = I.chi[c];
                Cs2[k] = I.C[c];
            }
        } else {
            gx3[q] = gy3[q] = ps3[q] = R(0);
            if (h2) rR2[k] = rB2[k] = jx2[k] = jy2[k] = a2[k] = ch2[k] = Cs2[k] = R(0);
        }
    }
    // (the tile meets a wall or mirror plane: block-uniform)
    const bool edge = __syncthreads_or(near_edge) != 0;
    lbfd2_tile<R, P, TX, TY>(I, ps, smem_raw, edge);
}

// ---------------------------------------------------------------------------
// Colour gradient and weights at t+1 from the moments of t+1 (set m), cell
// (x, y).
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ void grad2_next_cell(const Inst<R> &I, const MomSet<R> &m, int x,
                                                int y) {
    grad2_cell_from(I, x, y, m.rR, m.rB, m.rN);
}

// the same as its own launch (the SOR runs one launch a round), with the
// barrier counter of the one-launch form cleared
template <typename R>
__global__ void k_grad2n(Inst<R> I) {
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && threadIdx.y == 0)
        I.ctl->bar_count = 0;
    const MomSet<R> m = mom_of_step(I, I.ctl->step + 1);
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x < I.nx && y < I.ny) grad2_next_cell(I, m, x, y);
}

// ---------------------------------------------------------------------------
// k_sorfuse2: one cooperative launch per step after k_lbfd2.
//   1. colour gradient and weights at t+1 (grad2_next_cell), grid barrier;
//   2. SOR rounds: the blocked tiles of k_sor_tb2 (each block takes tiles
//      b, b + nblocks, ...), a grid barrier after each round, the same stop
//      decision in every block; a block also sums the surfactant of the
//      cells it stores (exact products, compensated sums) into its partial;
//   3. the total surfactant sum (a + eps) psi + (chi + eps) C of the result:
//      the partials of the last round, added by every block in the same
//      order;
//   4. rescale psi, C by M0 / total (Sec. 2.2) into the canonical buffers.
// Every barrier waits at most max_polls polls, then reports ST_TIMEOUT.
// ---------------------------------------------------------------------------
template <typename R, int TX, int TY, int K, int BS>
__global__ void __launch_bounds__(BS) k_sorfuse2(Inst<R> I, int max_rounds, long long max_polls) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const unsigned int nb = gridDim.x;
    const int tid = threadIdx.x;
    Ctl *ctl = I.ctl;
    const long long step0 = ctl->step;  // (block 0 advances it at the end)
    unsigned int bt = 0;                // arrivals that end the next grid barrier
    // the cells of this thread: every (nb BS)-th cell in row order from
    // b BS + tid, walked as (x, y) with the stride split once into (sx, sy)
    const long long stride = (long long)nb * BS;
    const int sx = int(stride % I.nx), sy = int(stride / I.nx);
    const long long q0 = (long long)blockIdx.x * BS + tid;
    const int x0 = int(q0 % I.nx), y0 = int(q0 / I.nx);
    // 1. gradient and weights of t+1
    const MomSet<R> mnext = mom_of_step(I, step0 + 1);
    for (int x = x0, y = y0; y < I.ny;) {
        grad2_next_cell(I, mnext, x, y);
        x += sx;
        y += sy;
        if (x >= I.nx) {
            x -= I.nx;
            y++;
        }
    }
    if (!grid_barrier(ctl, nb, bt, max_polls)) return;
    // 2. SOR rounds.  As a block stores its tiles' cells it also sums their
    //    surfactant; the round that ends the solve thus leaves the block
    //    partials of the total in I.part (3) with no pass of its own.
    const int tiles_x = (I.nx + TX - 1) / TX, tiles_y = (I.ny + TY - 1) / TY;
    const int nt = tiles_x * tiles_y;
    int round = 0;
    bool conv = false;
    if (I.transport) {
        for (;; round++) {
            R tsum[2] = {R(0), R(0)};
            for (int t = blockIdx.x; t < nt; t += nb) {
                if (t + (int)nb < nt)
                    sor_prefetch_tile<R, TX, TY, K, BS>(I, round, (t + nb) % tiles_x,
                                                        (t + nb) / tiles_x);
                sor_tile2<R, TX, TY, K, BS>(I, round, t % tiles_x, t / tiles_x, smem_raw, tsum,
                                            nt <= (int)nb);
            }
            double v[1] = {double(tsum[0]) + double(tsum[1])};
            double bsum[1];
            block_sum<BS, 1>(v, bsum);
            if (tid == 0) I.part[blockIdx.x] = bsum[0];
            if (!grid_barrier(ctl, nb, bt, max_polls)) return;
            conv = round_converged<R>(ctl, round, double(I.sor_tol));
            if (conv || round + 1 >= max_rounds) break;
        }
        round += 1;  // rounds run
    }
    // 3. total of the result: after `round` rounds it sits in the buffer the
    //    last round wrote
    const bool alt = ((round + I.sor_phase) & 1) != 0;
    const R *P = alt ? I.psi2 : I.psi;
    const R *Cq = alt ? I.C2 : I.C;
    if (!I.transport) {
        // (no solve: the total of the current values in a pass of its own;
        // each product exact as hi + lo, the thread's sum compensated)
        R hi = R(0), lo = R(0);
        for (int x = x0, y = y0; y < I.ny;) {
            const long long c = (long long)y * I.pitch + x;
            comp_add_prod(hi, lo, __ldcg(&I.a[c]) + I.eps_w, __ldcg(&P[c]));
            comp_add_prod(hi, lo, __ldcg(&I.chi[c]) + I.eps_w, __ldcg(&Cq[c]));
            x += sx;
            y += sy;
            if (x >= I.nx) {
                x -= I.nx;
                y++;
            }
        }
        double v[1] = {double(hi) + double(lo)};
        double bsum[1];
        block_sum<BS, 1>(v, bsum);
        if (tid == 0) I.part[blockIdx.x] = bsum[0];
        if (!grid_barrier(ctl, nb, bt, max_polls)) return;
    }
    // every block adds the block partials in the same order
    double acc[1] = {0.0};
    for (unsigned int k = tid; k < nb; k += BS) acc[0] += __ldcg(&I.part[k]);
    double tot[1];
    block_sum<BS, 1>(acc, tot);
    __shared__ double s_tot;
    if (tid == 0) s_tot = tot[0];
    __syncthreads();
    const double total = s_tot;
    const double scale = total > 0 ? ctl->M0 / total : 1.0;
    const double dscale = scale - 1.0;
    const float dscale_f = float(dscale);
    // 4. rescale: x (1 + d), d = s - 1, rounded without bias (rescale_one)
    for (int x = x0, y = y0; y < I.ny;) {
        const long long c = (long long)y * I.pitch + x;
        const R p = __ldcg(&P[c]), r = __ldcg(&Cq[c]);
        I.psi[c] = rescale_one(p, dscale, dscale_f, rescale_key(c, 0, step0));
        I.C[c] = rescale_one(r, dscale, dscale_f, rescale_key(c, 1, step0));
        x += sx;
        y += sy;
        if (x >= I.nx) {
            x -= I.nx;
            y++;
        }
    }
    if (blockIdx.x != 0) return;
    // the SOR convergence slots of the next solve start at zero (every block
    // has read this solve's slots before it reached the last barrier)
    unsigned long long *sw = &ctl->sweep[0][0];
    for (int k = tid; k < KMAX_SWEEPS * 4; k += BS) sw[k] = 0ull;
    if (tid != 0) return;
    if (I.transport) {
        ctl->pre = total;
        ctl->scale = scale;
        ctl->dscale = dscale;
        ctl->dscale_f = float(dscale);
        if (!conv) ctl->status |= ST_NOCONV;
        if (!isfinite(total)) {
            ctl->status |= ST_DIVERGED;
            ctl->dead = 1;
        }
        ctl->sor_iters = round * K;
    }
    ctl->sor_iters_parity = 0;
    ctl->sor_exec = 0;
    ctl->step += 1;
}

}  // namespace lbs
