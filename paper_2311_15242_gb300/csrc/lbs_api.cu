// lbs_api.cu — C ABI of the coupled LB-FD solver (include/lbs.h): context
// lifecycle, device workspace layout, CUDA-graph capture of one time step,
// field import/export and diagnostics.
#include <cuda_runtime.h>

#include <cfloat>
#include <cstddef>
#include <cstdint>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "../../include/lbs.h"
#include "lbs_d3q19.cuh"
#include "lbs_internal.h"
#include "lbs_k2d.cuh"
#include "lbs_fused2.cuh"
#include "lbs_launch3.h"

using namespace lbs;

namespace {

constexpr int BX = 32, BY = 8, BS = BX * BY;

// the blocked SOR kernel of variant v (tile, sweeps and threads:
// sor_vtx / sor_vty / sor_vk / sor_vbs)
#define LBS_SORV(v) sor_vtx(v), sor_vty(v), sor_vk(v), sor_vbs(v)
template <typename R>
void *sor2_kernel(int v) {
    switch (v) {
    case 1: return (void *)k_sor_tb2<R, LBS_SORV(1)>;
    case 2: return (void *)k_sor_tb2<R, LBS_SORV(2)>;
    case 3: return (void *)k_sor_tb2<R, LBS_SORV(3)>;
    case 4: return (void *)k_sor_tb2<R, LBS_SORV(4)>;
    case 5: return (void *)k_sor_tb2<R, LBS_SORV(5)>;
    case 6: return (void *)k_sor_tb2<R, LBS_SORV(6)>;
    case 7: return (void *)k_sor_tb2<R, LBS_SORV(7)>;
    case 8: return (void *)k_sor_tb2<R, LBS_SORV(8)>;
    default: return (void *)k_sor_tb2<R, LBS_SORV(0)>;
    }
}
// the one-launch form (gradient, SOR rounds, total and rescale) of variant v
template <typename R>
void *sor2_coop_kernel(int v) {
    switch (v) {
    case 1: return (void *)k_sorfuse2<R, LBS_SORV(1)>;
    case 2: return (void *)k_sorfuse2<R, LBS_SORV(2)>;
    case 3: return (void *)k_sorfuse2<R, LBS_SORV(3)>;
    case 4: return (void *)k_sorfuse2<R, LBS_SORV(4)>;
    case 5: return (void *)k_sorfuse2<R, LBS_SORV(5)>;
    case 6: return (void *)k_sorfuse2<R, LBS_SORV(6)>;
    case 7: return (void *)k_sorfuse2<R, LBS_SORV(7)>;
    case 8: return (void *)k_sorfuse2<R, LBS_SORV(8)>;
    default: return (void *)k_sorfuse2<R, LBS_SORV(0)>;
    }
}
template <typename R>
size_t sor2_smem(int v) {
    switch (v) {
    case 1: return SorTile<R, LBS_SORV(1)>::smem_bytes();
    case 2: return SorTile<R, LBS_SORV(2)>::smem_bytes();
    case 3: return SorTile<R, LBS_SORV(3)>::smem_bytes();
    case 4: return SorTile<R, LBS_SORV(4)>::smem_bytes();
    case 5: return SorTile<R, LBS_SORV(5)>::smem_bytes();
    case 6: return SorTile<R, LBS_SORV(6)>::smem_bytes();
    case 7: return SorTile<R, LBS_SORV(7)>::smem_bytes();
    case 8: return SorTile<R, LBS_SORV(8)>::smem_bytes();
    default: return SorTile<R, LBS_SORV(0)>::smem_bytes();
    }
}
#undef LBS_SORV

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// host-side equilibrium of one colour at rest for the shift (App. A, Eq. 37)
void rest_eq9(double rho, double al, double *f) {
    double m[Q9] = {rho, rho * (-3.6 * al - 0.4), rho * (5.4 * al - 1.4), 0, 0, 0, 0, 0, 0};
    for (int i = 0; i < Q9; i++) {
        double s = 0;
        for (int j = 0; j < Q9; j++) s += double(m9(j, i)) * m[j] / double(mnorm9(j));
        f[i] = s;
    }
}

// the same for D3Q19 (Eq. 40 at u = 0 through the closed-form inverse)
void rest_eq19(double rho, double al, double *f) {
    double m[Q19];
    meq19<double>(rho, 0.0, 0.0, 0.0, al, m);
    minv19<double>(m, f);
}


void set_err(lbs_ctx *c, const char *fmt, ...) {
    if (!c) return;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->err, sizeof(c->err), fmt, ap);
    va_end(ap);
}

#define CK(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            set_err(ctx, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                    __LINE__);                                                          \
            return LBS_ECUDA;                                                           \
        }                                                                               \
    } while (0)

// layout of the device workspace
struct Layout {
    int pitch;
    long long plane;
    size_t pops_off, scal_off, flag_off, ctl_off, part_off, stage_off, total;
    int nblocks;
};

// scalar planes: 21 in 2D, 25 in 3D (z components of j, grad, u, F), then
// the 4 rest-population planes of fT, fM, gT, gM and the previous time
// level of psi and C
constexpr int kScal2 = 21, kScal3 = 25, kRest = 6;
constexpr int kCoef2 = 6;  // 2D SOR coefficient planes (faces and inverse diagonals)
constexpr int kNext2 = 5;  // 2D moments of t+1 written by the fused step (rho^R, rho^B, rho^N, j)
// tile of the fused 2D step (k_lbfd2): TX x TY cells, one thread a cell
constexpr int FTX = 32, FTY = 16;

template <typename R, typename P>
Layout layout_of(const lbs_params *p) {
    Layout L;
    const bool d3 = p->nz > 1;
    L.pitch = (int)align_up(p->nx, 32);
    L.plane = (long long)align_up((size_t)L.pitch * p->ny * p->nz, 128);
    size_t pb = (size_t)L.plane * sizeof(R);
    L.pops_off = 0;
    size_t pops = 4 * (size_t)(d3 ? Q19 : Q9) * (size_t)L.plane * sizeof(P);
    L.scal_off = pops;
    size_t scal = ((d3 ? kScal3 : kScal2) + kRest + (d3 ? 0 : kCoef2 + kNext2)) * pb;
    L.flag_off = align_up(L.scal_off + scal, 256);
    L.ctl_off = align_up(L.flag_off + 2 * (size_t)L.plane, 256);
    L.part_off = align_up(L.ctl_off + sizeof(Ctl), 256);
    L.nblocks = ((p->nx + BX - 1) / BX) * ((p->ny + BY - 1) / BY) * p->nz;
    L.stage_off = align_up(L.part_off + (size_t)L.nblocks * (NDIAG + 3) * sizeof(double), 256);
    size_t N = (size_t)p->nx * p->ny * p->nz;
    L.total = align_up(L.stage_off + 12 * N * sizeof(double), 256);
    return L;
}

template <typename R, typename P>
struct Solver : Base {
    lbs_ctx *ctx;
    Inst<R> I;
    Layout L;
    char *ws;
    double *stage;
    cudaGraphExec_t gexec = nullptr;
    cudaGraph_t graph = nullptr;
    dim3 grid, block, sor_grid, surf_grid, diag_grid;
    int diag_blocks = 0;
    int surf_blocks = 0;
    bool prof = false;
    cudaEvent_t ev[LBS_K_NGROUPS + 1] = {};
    bool ran[LBS_K_NGROUPS] = {};

    const int D, Q;

    Solver(lbs_ctx *c) : ctx(c), D(c->p.nz > 1 ? 3 : 2), Q(c->p.nz > 1 ? Q19 : Q9) {
        const lbs_params *p = &c->p;
        L = layout_of<R, P>(p);
        ws = (char *)c->ws;
        std::memset(&I, 0, sizeof(I));
        I.nx = p->nx;
        I.ny = p->ny;
        I.nz = p->nz;
        I.pitch = L.pitch;
        I.plane = L.plane;
        I.bbmask = 0;
        I.mvmask = 0;
        for (int a = 0; a < 3; a++) {
            I.wall[a] = p->wall[a];
            I.bbmask |= (p->wall[a] == 1) << a;
            bool moving = false;
            for (int b = 0; b < 3; b++) moving |= p->uw_lo[a][b] != 0 || p->uw_hi[a][b] != 0;
            I.mvmask |= (p->wall[a] == 1 && moving) << a;
            for (int b = 0; b < 3; b++) {
                I.uw_lo[a][b] = R(p->uw_lo[a][b]);
                I.uw_hi[a][b] = R(p->uw_hi[a][b]);
            }
            I.g[a] = R(p->g[a]);
        }
        I.rhoR0 = R(p->rhoR0);
        I.rhoB0 = R(p->rhoB0);
        I.inv_rhoR0 = R(1.0 / p->rhoR0);
        I.inv_rhoB0 = R(1.0 / p->rhoB0);
        I.inv_2muR = R(0.5 / p->muR0);
        I.inv_2muB = R(0.5 / p->muB0);
        I.alphaR = R(p->alphaR);
        I.alphaB = R(p->alphaB);
        // (c_s^k)^2 = (3/5)(1 - alpha^k) in 2D, (1/2)(1 - alpha^k) in 3D (App. A)
        const double cf = D == 2 ? 0.6 : 0.5;
        I.cs2R = R(cf * (1.0 - p->alphaR));
        I.cs2B = R(cf * (1.0 - p->alphaB));
        I.muR0 = R(p->muR0);
        I.muB0 = R(p->muB0);
        I.beta = R(p->beta);
        I.eps_n = R(p->eps_n);
        I.eps_w = R(p->eps_w);
        I.sigma0 = R(p->sigma0);
        I.sigma_min = R(p->sigma_min_ratio * p->sigma0);
        I.E0 = R(p->E0);
        I.psi_inf = R(p->psi_inf);
        double cmc = (p->eos == 0 && p->E0 > 0)
                         ? p->psi_inf * (1.0 - std::exp(-(1.0 - p->sigma_min_ratio) / p->E0))
                         : (sizeof(R) == 4 ? (double)FLT_MAX : DBL_MAX);
        I.cmc = R(cmc);
        I.eos = p->eos;
        I.source = p->source;
        I.transport = p->transport;
        I.Ds = R(p->Ds);
        I.Db = R(p->Db);
        I.ra = R(p->ra);
        I.rd = R(p->rd);
        I.omega = R(p->sor_omega);
        I.sor_tol = R(p->sor_tol);
        I.sor_max_iter = p->sor_max_iter;
        // FP16 population scale: 2^14 / (the power of two >= the heavier pure density)
        {
            double rmax = p->rhoR0 > p->rhoB0 ? p->rhoR0 : p->rhoB0, sc = 16384.0;
            while (rmax > 1.0 && sc > 1.0) {
                rmax *= 0.5;
                sc *= 0.5;
            }
            I.pscale = R(sc);
            I.pinv = R(1.0 / sc);
        }
        // rest states of the pure phases; their moving components agree when
        // rhoR0 (1 - alphaR) = rhoB0 (1 - alphaB) (Eq. 42); the blue ones are used
        double sB[Q19], sR[Q19];
        if (D == 2) {
            rest_eq9(p->rhoB0, p->alphaB, sB);
            rest_eq9(p->rhoR0, p->alphaR, sR);
        } else {
            rest_eq19(p->rhoB0, p->alphaB, sB);
            rest_eq19(p->rhoR0, p->alphaR, sR);
        }
        double mov = 0;
        for (int i = 0; i < Q; i++) {
            I.shift[i] = R(sB[i]);
            if (i) mov += double(I.shift[i]);
        }
        I.shift0[0] = R(sB[0]);
        I.shift0[1] = R(sR[0]);
        for (int f = 0; f < 2; f++) {
            double tot = mov + double(I.shift0[f]);
            I.rho_s[f] = R(tot);
            double rk = f ? p->rhoR0 : p->rhoB0, ak = f ? p->alphaR : p->alphaB;
            I.dsh[f] = R(tot - rk);
            double e1 = 0, e2 = 0;
            for (int i = 0; i < Q; i++) {
                double si = i ? double(I.shift[i]) : double(I.shift0[f]);
                e1 += double(D == 2 ? m9(1, i) : m19(4, i)) * si;
                e2 += double(D == 2 ? m9(2, i) : m19(16, i)) * si;
            }
            if (D == 2) {
                I.mcor1[f] = R(e1 - rk * (-3.6 * ak - 0.4));
                I.mcor2[f] = R(e2 - rk * (5.4 * ak - 1.4));
            } else {
                const double pk = rk * 0.5 * (1.0 - ak);
                I.mcor1[f] = R(e1 - 3.0 * pk);
                I.mcor2[f] = R(e2 - pk / 3.0);
            }
        }
        I.sor_pingpong = D == 2;  // (set by set_sor_grid)
        size_t pb = (size_t)L.plane;
        P *pops = (P *)(ws + L.pops_off);
        I.fT = pops;
        I.fM = pops + 1 * Q * pb;
        I.gT = pops + 2 * Q * pb;
        I.gM = pops + 3 * Q * pb;
        I.flag = (uint8_t *)(ws + L.flag_off);
        I.gflag = I.flag + L.plane;
        R *sc = (R *)(ws + L.scal_off);
        R **fields[] = {&I.rhoR, &I.rhoB, &I.rhoN, &I.jx,  &I.jy,  &I.gx,  &I.gy,
                        &I.a,    &I.chi,  &I.ux,   &I.uy,  &I.Fx,  &I.Fy,  &I.psi,
                        &I.C,    &I.S,    &I.B,    &I.rpsi, &I.rC, &I.psi2, &I.C2};
        for (int k = 0; k < kScal2; k++) *fields[k] = sc + k * pb;
        if (D == 3) {
            R **f3[] = {&I.jz, &I.gz, &I.uz, &I.Fz};
            for (int k = 0; k < kScal3 - kScal2; k++) *f3[k] = sc + (kScal2 + k) * pb;
        }
        {
            R **fr[] = {&I.fT0, &I.fM0, &I.gT0, &I.gM0, &I.psip, &I.Cp};
            const int base = D == 3 ? kScal3 : kScal2;
            for (int k = 0; k < kRest; k++) *fr[k] = sc + (base + k) * pb;
        }
        if (D == 2) {
            R **fc[] = {&I.sfx, &I.sfy, &I.scx, &I.scy, &I.sip, &I.sic};
            for (int k = 0; k < kCoef2; k++) *fc[k] = sc + (kScal2 + kRest + k) * pb;
            R **fn[] = {&I.rhoRn, &I.rhoBn, &I.rhoNn, &I.jxn, &I.jyn};
            for (int k = 0; k < kNext2; k++) *fn[k] = sc + (kScal2 + kRest + kCoef2 + k) * pb;
            // the fused step: populations alternate between the two sets, the
            // solve starts from the guess in the second buffers
            I.pop_pp = 1;
            I.sor_phase = 1;
        }
        I.ctl = (Ctl *)(ws + L.ctl_off);
        I.part = (double *)(ws + L.part_off);
        stage = (double *)(ws + L.stage_off);
        block = dim3(BX, BY, 1);
        grid = dim3((p->nx + BX - 1) / BX, (p->ny + BY - 1) / BY, p->nz);
        set_sor_grid();
        const long long rows = (long long)p->ny * p->nz;
        surf_grid = dim3((p->nx + BX - 1) / BX,
                         (unsigned)((rows + BY * SURF_STRIP - 1) / (BY * SURF_STRIP)), 1);
        surf_blocks = (int)(surf_grid.x * surf_grid.y);
        diag_grid = dim3(grid.x, (p->ny + BY * DIAG_STRIP - 1) / (BY * DIAG_STRIP), p->nz);
        diag_blocks = (int)(diag_grid.x * diag_grid.y * diag_grid.z);
        for (int v = 0; v < kSorVariants; v++)
            if (sor2_fits(v)) {
                cudaFuncSetAttribute(sor2_kernel<R>(v),
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)sor2_smem<R>(v));
                cudaFuncSetAttribute(sor2_coop_kernel<R>(v),
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)sor2_smem<R>(v));
            }
        if (D == 3)
            cudaFuncSetAttribute(Launch3<R, P>::zm_fn(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)Launch3<R, P>::zm_smem());
        if (D == 2) {
            cudaFuncSetAttribute(k_lbfd2<R, P, FTX, FTY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)Fuse2<R, FTX, FTY>::bytes());
            fgrid = dim3((p->nx + FTX - 1) / FTX, (p->ny + FTY - 1) / FTY, 1);
        }
    }
    dim3 fgrid;  // tiles of the fused 2D step

    // SOR variant: 2D the blocked tile (sor_vtx ...); 3D 0 = red-black
    // half-sweeps in place, 1 = z-marching full sweeps (ping-pong buffers),
    // 2, 3 = red-black half-sweeps in place by column marching (8 or 4 planes)
    int sv = 0;
    void set_sor_grid() {
        using L3 = Launch3<R, P>;
        if (D == 2) {
            sor_grid = dim3((I.nx + sor_vtx(sv) - 1) / sor_vtx(sv),
                            (I.ny + sor_vty(sv) - 1) / sor_vty(sv), 1);
        } else if (sv == 1) {
            sor_grid = L3::zm_grid(I.nx, I.ny, I.nz);
        } else {
            // red-black half-sweeps: one thread per cell pair along x (and per
            // plane, or per chunk of planes when column marching)
            sor_grid = L3::sor_grid(sv, I.nx, I.ny, I.nz);
        }
        I.sor_pingpong = (D == 2 || sv == 1) ? 1 : 0;
        coop_ok = false;
        if (D == 2) {
            // one launch for all rounds (k_sorfuse2): as many blocks as are
            // resident at once, up to one a tile; each block takes tiles b,
            // b + blocks, ... in every round
            int dev = 0, sms = 0, coop = 0, per_sm = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
            if (sor2_fits(sv))
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sor2_coop_kernel<R>(sv),
                                                              sor_vbs(sv), sor2_smem<R>(sv));
            const long long tiles = (long long)sor_grid.x * sor_grid.y;
            const long long resident = (long long)per_sm * sms;
            coop_blocks = (int)(tiles < resident ? tiles : resident);
            coop_ok = coop && coop_blocks > 0;
        }
    }
    int coop_blocks = 0;  // blocks of the one-launch form
    bool coop_ok = false;  // the one-launch SOR applies to this grid and variant
    bool coop_on = true;   // and is wanted (lbs_set_sor_persistent)
    bool use_coop() const { return D == 2 && coop_ok && coop_on; }
    long long coop_polls = kBarrierPolls;  // the barrier's wait limit
    int set_sor_wait_limit(long long polls) override {
        if (polls < 0) {
            set_err(ctx, "wait limit must be >= 0 polls");
            return LBS_EINVAL;
        }
        CK(cudaStreamSynchronize(ctx->stream));
        coop_polls = polls;
        if (gexec) {
            CK(cudaGraphExecDestroy(gexec));
            CK(cudaGraphDestroy(graph));
            gexec = nullptr;
            graph = nullptr;
        }
        return LBS_OK;
    }
    int set_sor_persistent(int on) override {
        CK(cudaStreamSynchronize(ctx->stream));
        coop_on = on != 0;
        if (gexec) {
            CK(cudaGraphExecDestroy(gexec));
            CK(cudaGraphDestroy(graph));
            gexec = nullptr;
            graph = nullptr;
        }
        return LBS_OK;
    }
    // the gradient, all rounds of the solve, the total and the rescale in one
    // cooperative launch (k_sorfuse2)
    int launch_sor_coop(cudaStream_t s) {
        int maxr = sor_rounds();
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(coop_blocks, 1, 1);
        cfg.blockDim = dim3(sor_vbs(sv), 1, 1);
        cfg.dynamicSmemBytes = sor2_smem<R>(sv);
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeCooperative;
        at[0].val.cooperative = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        long long polls = coop_polls;
        void *args[] = {(void *)&I, (void *)&maxr, (void *)&polls};
        CK(cudaLaunchKernelExC(&cfg, sor2_coop_kernel<R>(sv), args));
        return LBS_OK;
    }
    // variant v's shared memory fits a block on this device
    static bool sor2_fits(int v) {
        int dev = 0, lim = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&lim, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        return sor2_smem<R>(v) <= (size_t)lim;
    }
    int set_sor_tile(int v) override {
        if (v < 0 || v >= (D == 2 ? kSorVariants : 4)) {
            set_err(ctx, "SOR variant %d: 0..%d in 2D, 0..3 in 3D", v, kSorVariants - 1);
            return LBS_EINVAL;
        }
        if (D == 2 && !sor2_fits(v)) {
            set_err(ctx, "SOR variant %d needs %zu bytes of shared memory a block in this "
                         "storage form", v, sor2_smem<R>(v));
            return LBS_EINVAL;
        }
        CK(cudaStreamSynchronize(ctx->stream));
        sv = v;
        set_sor_grid();
        if (gexec) {
            CK(cudaGraphExecDestroy(gexec));
            CK(cudaGraphDestroy(graph));
            gexec = nullptr;
            graph = nullptr;
        }
        return LBS_OK;
    }

    ~Solver() {
        if (gexec) cudaGraphExecDestroy(gexec);
        if (graph) cudaGraphDestroy(graph);
        for (auto &e : ev)
            if (e) cudaEventDestroy(e);
    }

    // (recorded as an event node when captured into the step graph)
    // (a group ends at the next mark recorded in the same step)
    bool marked[LBS_K_NGROUPS + 1] = {};
    void mark(cudaStream_t s, int g) {
        if (!prof) return;
        marked[g] = true;
        if (capturing)
            cudaEventRecordWithFlags(ev[g], s, cudaEventRecordExternal);
        else
            cudaEventRecord(ev[g], s);
    }
    bool capturing = false;
    bool use_graph = true;

    int launch_check() {
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            set_err(ctx, "kernel launch failed: %s", cudaGetErrorString(e));
            return LBS_ECUDA;
        }
        return LBS_OK;
    }

    // the launches of one time step, in order, captured into the step graph;
    // with profiling on, an event is recorded at every group boundary.  The
    // SOR rounds run in one cooperative launch (2D, when the grid fits the
    // device at once), else in a WHILE conditional node whose body is one
    // round, whose last block ends the loop on convergence.
    int capture_step(cudaStream_t s, cudaGraph_t g) {
        CK(cudaStreamBeginCaptureToGraph(s, g, nullptr, nullptr, 0,
                                         cudaStreamCaptureModeThreadLocal));
        capturing = true;
        int r = enqueue_step(s);
        capturing = false;
        cudaGraph_t out = nullptr;
        cudaError_t e = cudaStreamEndCapture(s, &out);
        if (r) return r;
        if (e != cudaSuccess) {
            set_err(ctx, "graph capture failed: %s", cudaGetErrorString(e));
            return LBS_ECUDA;
        }
        return LBS_OK;
    }

    // launches of one step; the one-launch SOR is the same launch in a capture
    // and outside it; otherwise, inside a capture the SOR loop becomes the
    // WHILE node, outside it a host loop of sor_rounds() launches that return
    // at once after the round that converged
    using L3 = Launch3<R, P>;
    void k_force(cudaStream_t s) {
        if (D == 2)
            k_force2<R><<<grid, block, 0, s>>>(I);
        else
            L3::force(I, grid, block, s);
    }

    // a kernel that directly follows another kernel of the step (no event or
    // conditional node between them) launches as its programmatic dependent:
    // it starts while that kernel's last blocks run and waits (pdl_wait) for
    // its completion before touching any field.  With profiling events
    // between the groups, an ordinary launch.
    template <typename... K, typename... A>
    void launch_dep(void (*k)(K...), dim3 g, dim3 b, cudaStream_t s, A... args) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = g;
        cfg.blockDim = b;
        cfg.dynamicSmemBytes = 0;
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = at;
        cfg.numAttrs = prof ? 0 : 1;
        cudaLaunchKernelEx(&cfg, k, args...);
    }

    int enqueue_step(cudaStream_t s) {
        for (bool &r : ran) r = false;
        for (bool &m : marked) m = false;
        if (D == 2) {
            // the fused step: force, surfactant terms, collision, recolouring
            // and streaming in one launch (timed as the collide group) ...
            mark(s, LBS_K_COLLIDE);
            k_lbfd2<R, P, FTX, FTY><<<fgrid, FTX * FTY, Fuse2<R, FTX, FTY>::bytes(), s>>>(I);
            ran[LBS_K_COLLIDE] = true;
            if (I.transport && use_coop()) {
                // ... then the gradient, every SOR round, the total and the
                // rescale in one cooperative launch (timed as the SOR group)
                mark(s, LBS_K_SOR);
                int r = launch_sor_coop(s);
                if (r) return r;
                ran[LBS_K_SOR] = true;
                mark(s, LBS_K_NGROUPS);
                return launch_check();
            }
            // ... or the gradient, one launch a round and the total and
            // rescale as launches of their own
            mark(s, LBS_K_GRAD);
            launch_dep(k_grad2n<R>, grid, block, s, I);
            ran[LBS_K_GRAD] = true;
        } else {
            mark(s, LBS_K_FORCE);
            k_force(s);
            ran[LBS_K_FORCE] = true;
            mark(s, LBS_K_FD);
            if (I.transport) {
                L3::fd(I, grid, block, s, nullptr, nullptr);
                ran[LBS_K_FD] = true;
            }
            mark(s, LBS_K_COLLIDE);
            L3::collide(I, grid, block, s);
            ran[LBS_K_COLLIDE] = true;
            mark(s, LBS_K_STREAM);
            L3::stream(I, grid, block, s);
            ran[LBS_K_STREAM] = true;
            mark(s, LBS_K_GRAD);
            L3::grad(I, grid, block, s);
            ran[LBS_K_GRAD] = true;
        }
        mark(s, LBS_K_SOR);
        if (I.transport && !capturing) {
            // eager form (for profilers): the host reads the loop state after
            // every round and launches no round beyond the converged one
            for (int r = 0; r < sor_rounds(); r++) {
                launch_sor_round(s, cudaGraphConditionalHandle(0), r);
                int done = 0;
                CK(cudaMemcpyAsync(&done, &I.ctl->sor_exec, sizeof(int), cudaMemcpyDeviceToHost, s));
                CK(cudaStreamSynchronize(s));
                if (done < 0) break;
            }
            ran[LBS_K_SOR] = true;
        } else if (I.transport) {
            cudaStreamCaptureStatus st;
            cudaGraph_t cg;
            const cudaGraphNode_t *deps = nullptr;
            size_t nd = 0;
            CK(cudaStreamGetCaptureInfo(s, &st, nullptr, &cg, &deps, nullptr, &nd));
            cudaGraphConditionalHandle h;
            CK(cudaGraphConditionalHandleCreate(&h, cg, 1, cudaGraphCondAssignDefault));
            cudaGraphNodeParams cp = {};
            cp.type = cudaGraphNodeTypeConditional;
            cp.conditional.handle = h;
            cp.conditional.type = cudaGraphCondTypeWhile;
            cp.conditional.size = 1;
            cudaGraphNode_t cnode;
            CK(cudaGraphAddNode(&cnode, cg, deps, nullptr, nd, &cp));
            cudaGraph_t body = cp.conditional.phGraph_out[0];
            int maxr = sor_rounds(), eager = -1;
            if (D == 2) {
                void *args[] = {(void *)&I, (void *)&h, (void *)&maxr, (void *)&eager};
                cudaKernelNodeParams kp = {};
                kp.func = sor2_kernel<R>(sv);
                kp.gridDim = sor_grid;
                kp.blockDim = dim3(sor_vbs(sv), 1, 1);
                kp.sharedMemBytes = (unsigned)sor2_smem<R>(sv);
                kp.kernelParams = args;
                cudaGraphNode_t kn;
                CK(cudaGraphAddKernelNode(&kn, body, nullptr, 0, &kp));
            } else if (sv == 1) {
                // body: one z-marching sweep
                void *args[] = {(void *)&I, (void *)&h, (void *)&maxr, (void *)&eager};
                cudaKernelNodeParams kp = {};
                kp.func = L3::zm_fn();
                kp.gridDim = sor_grid;
                kp.blockDim = dim3(L3::zm_threads(), 1, 1);
                kp.sharedMemBytes = (unsigned)L3::zm_smem();
                kp.kernelParams = args;
                cudaGraphNode_t kn;
                CK(cudaGraphAddKernelNode(&kn, body, nullptr, 0, &kp));
            } else {
                // body: red half-sweep, then black half-sweep
                cudaGraphNode_t kn[2];
                for (int colour = 0; colour < 2; colour++) {
                    int col = colour;
                    void *args[] = {(void *)&I, (void *)&col, (void *)&h, (void *)&maxr,
                                    (void *)&eager};
                    cudaKernelNodeParams kp = {};
                    kp.func = L3::sor_fn(sv);
                    kp.gridDim = sor_grid;
                    kp.blockDim = dim3(L3::kSorBX, L3::kSorBY, 1);
                    kp.sharedMemBytes = 0;
                    kp.kernelParams = args;
                    CK(cudaGraphAddKernelNode(&kn[colour], body, colour ? &kn[0] : nullptr,
                                              colour ? 1 : 0, &kp));
                }
            }
            CK(cudaStreamUpdateCaptureDependencies(s, &cnode, nullptr, 1,
                                                   cudaStreamSetCaptureDependencies));
            ran[LBS_K_SOR] = true;
        }
        mark(s, LBS_K_SURF);
        if (I.transport) {
            k_surf2<R, BS><<<surf_grid, block, 0, s>>>(I, 1, surf_blocks, sweeps_per_round());
            if (D == 2)
                launch_dep(k_scale2<R>, grid, block, s, I);
            else
                k_scale2<R><<<grid, block, 0, s>>>(I);
        } else {
            k_tick<R><<<1, 32, 0, s>>>(I);
        }
        ran[LBS_K_SURF] = true;
        mark(s, LBS_K_NGROUPS);
        return launch_check();
    }

    // one SOR round outside a graph (eager mode): 2D one blocked launch of K
    // sweeps, 3D a red and a black half-sweep
    void launch_sor_round(cudaStream_t s, cudaGraphConditionalHandle h, int r) {
        if (D == 2) {
            int maxr = sor_rounds();
            void *args[] = {(void *)&I, (void *)&h, (void *)&maxr, (void *)&r};
            cudaLaunchKernel(sor2_kernel<R>(sv), sor_grid, dim3(sor_vbs(sv)), args, sor2_smem<R>(sv),
                             s);
        } else if (sv == 1) {
            int maxr = sor_rounds();
            void *args[] = {(void *)&I, (void *)&h, (void *)&maxr, (void *)&r};
            cudaLaunchKernel(L3::zm_fn(), sor_grid, dim3(L3::zm_threads()), args, L3::zm_smem(), s);
        } else {
            const dim3 b(L3::kSorBX, L3::kSorBY, 1);
            L3::sor(I, sor_grid, b, s, 0, h, sor_rounds(), r, sv);
            L3::sor(I, sor_grid, b, s, 1, h, sor_rounds(), r, sv);
        }
    }

    int sweeps_per_round() const { return D == 2 ? sor_vk(sv) : 1; }

    int step_result(double *out) override {
        int r = sync();
        if (r) return r;
        struct {
            long long step;
            double M0, pre, scale;
        } h;
        static_assert(offsetof(Ctl, step) == 0 && offsetof(Ctl, scale) == 3 * sizeof(double),
                      "control block layout");
        CK(cudaMemcpy(&h, I.ctl, sizeof(h), cudaMemcpyDeviceToHost));
        out[0] = double(h.step);
        out[1] = h.pre;
        out[2] = h.scale;
        return LBS_OK;
    }

    // ---- checkpoint: the state that carries from one step to the next ----
    // every plane a step reads before writing it: the moving populations
    // (storage type) and the rest populations of the current set, the flags,
    // the moments, colour gradient and weights of the current time level,
    // u and F, psi and C, the Adams-Bashforth history S, B (Eqs. 23-24) and
    // the previous time level psip, Cp of the SOR starting guess
    struct Plane {
        void *d;
        size_t es;
    };
    // (step: the saved or loaded step counter; the fused 2D step keeps the
    // populations of step s in set s & 1)
    int state_planes(Plane *out, long long step) const {
        const bool odd = I.pop_pp && (step & 1);
        void *T = odd ? I.gT : I.fT, *M = odd ? I.gM : I.fM;
        R *T0 = odd ? I.gT0 : I.fT0, *M0 = odd ? I.gM0 : I.fM0;
        uint8_t *fl = odd ? I.gflag : I.flag;
        int n = 0;
        for (int i = 1; i < Q; i++)
            out[n++] = {(char *)T + (size_t)i * L.plane * sizeof(P), sizeof(P)};
        for (int i = 1; i < Q; i++)
            out[n++] = {(char *)M + (size_t)i * L.plane * sizeof(P), sizeof(P)};
        const MomSet<R> m = mom_set(I, odd);
        R *const sc[] = {T0,    M0,    m.rR, m.rB, m.rN, m.jx, m.jy, I.gx, I.gy, I.a,
                         I.chi, I.ux,  I.uy, I.Fx, I.Fy, I.psi, I.C, I.S, I.B, I.psip, I.Cp};
        for (R *f : sc) out[n++] = {f, sizeof(R)};
        if (D == 3) {
            R *const s3[] = {I.jz, I.gz, I.uz, I.Fz};
            for (R *f : s3) out[n++] = {f, sizeof(R)};
        }
        out[n++] = {fl, 1};
        return n;
    }
    static constexpr uint32_t kStateMagic = 0x5453424cu;  // "LBST"
    static constexpr uint32_t kStateVersion = 1;
    struct StateHeader {
        uint32_t magic, version;
        int32_t nx, ny, nz, storage, r_bytes, p_bytes, nplanes, sor_iters, sor_iters_parity, pad;
        long long step;
        double M0, pre, scale, dscale;
        float dscale_f, pad_f;
        unsigned long long total;
    };
    size_t state_bytes() const {
        Plane pl[2 * Q19 + 32];
        const int n = state_planes(pl, 0);
        const size_t N = (size_t)I.nx * I.ny * I.nz;
        size_t b = sizeof(StateHeader);
        for (int k = 0; k < n; k++) b += N * pl[k].es;
        return b;
    }
    int save_state(void *buf, size_t *bytes) override {
        const size_t need = state_bytes();
        if (!buf) {
            *bytes = need;
            return LBS_OK;
        }
        if (*bytes < need) {
            set_err(ctx, "state buffer of %zu bytes (need %zu)", *bytes, need);
            *bytes = need;
            return LBS_EINVAL;
        }
        int r = sync();
        if (r) return r;
        cudaStream_t s = ctx->stream;
        Ctl h;
        CK(cudaMemcpy(&h, I.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
        Plane pl[2 * Q19 + 32];
        const int n = state_planes(pl, h.step);
        StateHeader hd;
        std::memset(&hd, 0, sizeof(hd));
        hd.magic = kStateMagic;
        hd.version = kStateVersion;
        hd.nx = I.nx;
        hd.ny = I.ny;
        hd.nz = I.nz;
        hd.storage = ctx->storage;
        hd.r_bytes = (int)sizeof(R);
        hd.p_bytes = (int)sizeof(P);
        hd.nplanes = n;
        hd.sor_iters = h.sor_iters;
        hd.sor_iters_parity = h.sor_iters_parity;
        hd.step = h.step;
        hd.M0 = h.M0;
        hd.pre = h.pre;
        hd.scale = h.scale;
        hd.dscale = h.dscale;
        hd.dscale_f = h.dscale_f;
        hd.total = need;
        std::memcpy(buf, &hd, sizeof(hd));
        char *o = (char *)buf + sizeof(hd);
        const size_t rows = (size_t)I.ny * I.nz;
        for (int k = 0; k < n; k++) {
            const size_t w = (size_t)I.nx * pl[k].es;
            CK(cudaMemcpy2DAsync(o, w, pl[k].d, (size_t)I.pitch * pl[k].es, w, rows,
                                 cudaMemcpyDeviceToHost, s));
            o += w * rows;
        }
        CK(cudaStreamSynchronize(s));
        *bytes = need;
        return LBS_OK;
    }
    int load_state(const void *buf, size_t bytes) override {
        StateHeader hd;
        if (bytes < sizeof(hd)) {
            set_err(ctx, "state buffer of %zu bytes is shorter than its header", bytes);
            return LBS_EINVAL;
        }
        std::memcpy(&hd, buf, sizeof(hd));
        Plane pl[2 * Q19 + 32];
        const int n = state_planes(pl, hd.step);
        if (hd.magic != kStateMagic || hd.version != kStateVersion) {
            set_err(ctx, "not a saved state of this library version");
            return LBS_EINVAL;
        }
        if (hd.nx != I.nx || hd.ny != I.ny || hd.nz != I.nz || hd.storage != ctx->storage ||
            hd.r_bytes != (int)sizeof(R) || hd.p_bytes != (int)sizeof(P) || hd.nplanes != n) {
            set_err(ctx, "saved state is %dx%dx%d storage %d; this context is %dx%dx%d storage %d",
                    hd.nx, hd.ny, hd.nz, hd.storage, I.nx, I.ny, I.nz, ctx->storage);
            return LBS_EINVAL;
        }
        if (hd.total != state_bytes() || bytes < hd.total) {
            set_err(ctx, "saved state of %zu bytes, expected %zu", bytes, state_bytes());
            return LBS_EINVAL;
        }
        cudaStream_t s = ctx->stream;
        CK(cudaStreamSynchronize(s));
        const char *o = (const char *)buf + sizeof(hd);
        const size_t rows = (size_t)I.ny * I.nz;
        for (int k = 0; k < n; k++) {
            const size_t w = (size_t)I.nx * pl[k].es;
            CK(cudaMemcpy2DAsync(pl[k].d, (size_t)I.pitch * pl[k].es, o, w, w, rows,
                                 cudaMemcpyHostToDevice, s));
            o += w * rows;
        }
        // the control block: counters and totals of the saved step; status,
        // arrival counters and SOR progress start clear
        Ctl h;
        std::memset(&h, 0, sizeof(h));
        h.step = hd.step;
        h.M0 = hd.M0;
        h.pre = hd.pre;
        h.scale = hd.scale;
        h.dscale = hd.dscale;
        h.dscale_f = hd.dscale_f;
        h.sor_iters = hd.sor_iters;
        h.sor_iters_parity = hd.sor_iters_parity;
        CK(cudaMemcpyAsync(I.ctl, &h, sizeof(Ctl), cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));
        return LBS_OK;
    }

    const void *inst() const override { return &I; }
    size_t inst_bytes() const override { return sizeof(I); }
    void set_batch_member() override {
        I.pop_pp = 0;
        I.sor_phase = 0;
    }

    int set_graph(int on) override {
        use_graph = bool(on);
        return LBS_OK;
    }

    int sor_rounds() const {
        return (I.sor_max_iter + sweeps_per_round() - 1) / sweeps_per_round();
    }

    // kernels of one step with the SOR loop at the round count of the last
    // diagnostics (4 before the first): one launch a round, two for the 3D
    // red-black half-sweeps
    int kernel_count() const override {
        if (D == 2 && I.transport && use_coop()) return 2;
        const int per_round = (D == 3 && sv != 1) ? 2 : 1;
        const int cells = D == 2 ? 2 : 5;  // 2D: the fused step and the gradient
        return I.transport ? cells + 2 + per_round * last_rounds : cells + 1;
    }
    int last_rounds = 4;

    int profile(int on) override {
        if (bool(on) == prof) return LBS_OK;
        if (on)
            for (auto &e : ev)
                if (!e) CK(cudaEventCreate(&e));
        prof = bool(on);
        if (gexec) {  // rebuild with / without the event nodes
            CK(cudaGraphExecDestroy(gexec));
            CK(cudaGraphDestroy(graph));
            gexec = nullptr;
            graph = nullptr;
        }
        return LBS_OK;
    }

    int kernel_times(double *ms, int n) override {
        if (!prof) {
            set_err(ctx, "profiling is off (lbs_profile)");
            return LBS_EINVAL;
        }
        CK(cudaStreamSynchronize(ctx->stream));
        for (int g = 0; g < n && g < LBS_K_NGROUPS; g++) {
            float t = 0;
            int h = g + 1;
            while (h < LBS_K_NGROUPS && !marked[h]) h++;
            if (ran[g] && marked[g]) CK(cudaEventElapsedTime(&t, ev[g], ev[h]));
            ms[g] = t;
        }
        return LBS_OK;
    }

    int init(const double *phi, const double *psi, const double *C, const double *u) override {
        size_t N = (size_t)I.nx * I.ny * I.nz;
        cudaStream_t s = ctx->stream;
        double *dphi = stage, *dpsi = stage + N, *dC = stage + 2 * N, *du = stage + 3 * N;
        CK(cudaMemcpyAsync(dphi, phi, N * sizeof(double), cudaMemcpyHostToDevice, s));
        if (psi) CK(cudaMemcpyAsync(dpsi, psi, N * sizeof(double), cudaMemcpyHostToDevice, s));
        if (C) CK(cudaMemcpyAsync(dC, C, N * sizeof(double), cudaMemcpyHostToDevice, s));
        if (u) CK(cudaMemcpyAsync(du, u, 3 * N * sizeof(double), cudaMemcpyHostToDevice, s));
        CK(cudaMemsetAsync(ws + L.pops_off, 0, L.ctl_off - L.pops_off, s));
        CK(cudaMemsetAsync(I.ctl, 0, sizeof(Ctl), s));
        if (D == 2) {
            k_init2<R, P><<<grid, block, 0, s>>>(I, dphi, psi ? dpsi : nullptr,
                                              C ? dC : nullptr, u ? du : nullptr);
            k_moments2<R, P><<<grid, block, 0, s>>>(I);
            k_grad2<R><<<grid, block, 0, s>>>(I, 0);
        } else {
            L3::init(I, grid, block, s, dphi, psi ? dpsi : nullptr, C ? dC : nullptr,
                     u ? du : nullptr);
            L3::moments(I, grid, block, s);
            L3::grad(I, grid, block, s, 0);
        }
        k_surf2<R, BS><<<surf_grid, block, 0, s>>>(I, 0, surf_blocks, sweeps_per_round());
        int r = launch_check();
        if (r) return r;
        CK(cudaStreamSynchronize(s));
        return LBS_OK;
    }

    int build_graph() {
        CK(cudaGraphCreate(&graph, 0));
        int r = capture_step(ctx->stream, graph);
        if (r) return r;
        CK(cudaGraphInstantiate(&gexec, graph, 0));
        return LBS_OK;
    }

    int step(int n) override {
        if (n <= 0) return LBS_OK;
        if (!use_graph) {
            for (int k = 0; k < n; k++) {
                int r = enqueue_step(ctx->stream);
                if (r) return r;
            }
            return LBS_OK;
        }
        if (!gexec) {
            int r = build_graph();
            if (r) return r;
        }
        for (int k = 0; k < n; k++) CK(cudaGraphLaunch(gexec, ctx->stream));
        return LBS_OK;
    }

    int sync() override {
        CK(cudaStreamSynchronize(ctx->stream));
        int st = 0;
        CK(cudaMemcpy(&st, &I.ctl->status, sizeof(int), cudaMemcpyDeviceToHost));
        if (st) {
            int zero = 0;
            CK(cudaMemcpy(&I.ctl->status, &zero, sizeof(int), cudaMemcpyHostToDevice));
            if (st & ST_DIVERGED) {
                set_err(ctx, "non-finite total surfactant (diverged)");
                return LBS_EDIVERGED;
            }
            if (st & ST_TIMEOUT) {
                set_err(ctx, "a bounded device wait gave up");
                return LBS_ETIMEOUT;
            }
            if (st & ST_NOCONV) {
                set_err(ctx, "SOR did not converge within %d sweeps", I.sor_max_iter);
                return LBS_ENOCONV;
            }
        }
        return LBS_OK;
    }

    int get(double *rho, double *u, double *phi, double *psi, double *C) override {
        int r = sync();
        if (r) return r;
        size_t N = (size_t)I.nx * I.ny * I.nz;
        cudaStream_t s = ctx->stream;
        k_force(s);
        k_export2<R><<<grid, block, 0, s>>>(I, stage, stage + N, stage + 4 * N, stage + 5 * N,
                                            stage + 6 * N);
        r = launch_check();
        if (r) return r;
        if (rho) CK(cudaMemcpyAsync(rho, stage, N * sizeof(double), cudaMemcpyDeviceToHost, s));
        if (u) CK(cudaMemcpyAsync(u, stage + N, 3 * N * sizeof(double), cudaMemcpyDeviceToHost, s));
        if (phi) CK(cudaMemcpyAsync(phi, stage + 4 * N, N * sizeof(double), cudaMemcpyDeviceToHost, s));
        if (psi) CK(cudaMemcpyAsync(psi, stage + 5 * N, N * sizeof(double), cudaMemcpyDeviceToHost, s));
        if (C) CK(cudaMemcpyAsync(C, stage + 6 * N, N * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        return LBS_OK;
    }

    int macro(double *g, double *a, double *F, double *u, double *S, double *B) override {
        int r = sync();
        if (r) return r;
        size_t N = (size_t)I.nx * I.ny * I.nz;
        cudaStream_t s = ctx->stream;
        k_force(s);
        double *dg = stage, *da = stage + 3 * N, *dF = stage + 4 * N, *du = stage + 7 * N,
               *dS = stage + 10 * N, *dB = stage + 11 * N;
        k_export_macro2<R><<<grid, block, 0, s>>>(I, dg, da, dF, du);
        if (D == 2)
            k_fd2<R><<<grid, block, 0, s>>>(I, dS, dB);
        else
            L3::fd(I, grid, block, s, dS, dB);
        r = launch_check();
        if (r) return r;
        struct {
            double *h, *d;
            size_t n;
        } cp[] = {{g, dg, 3 * N}, {a, da, N}, {F, dF, 3 * N}, {u, du, 3 * N}, {S, dS, N}, {B, dB, N}};
        for (auto &c : cp)
            if (c.h) CK(cudaMemcpyAsync(c.h, c.d, c.n * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        return LBS_OK;
    }

    int diag(lbs_diag *d) override {
        int r = sync();
        if (r) return r;
        cudaStream_t s = ctx->stream;
        k_force(s);
        if (D == 2)
            k_diag<R, P, BS, Q9><<<diag_grid, block, 0, s>>>(I, diag_blocks);
        else
            L3::diag(I, diag_grid, block, s, diag_blocks);
        r = launch_check();
        if (r) return r;
        Ctl h;
        CK(cudaMemcpyAsync(&h, I.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        const double *v = h.diag;
        std::memset(d, 0, sizeof(*d));
        d->mass_R = v[0];
        d->mass_B = v[1];
        d->surf_total = v[2];
        d->surf_pre_rescale = h.pre;
        d->rescale_factor = h.scale;
        const lbs_params *p = &ctx->p;
        int D = p->nz == 1 ? 2 : 3;
        int vert = D - 1;
        double gmax = 0;
        for (int a = 0; a < D; a++)
            if (std::fabs(p->g[a]) > gmax) {
                gmax = std::fabs(p->g[a]);
                vert = a;
            }
        double cnt = v[3];
        if (cnt > 0) {
            d->U[0] = v[4] / cnt;
            d->U[1] = v[5] / cnt;
            d->U[2] = v[15] / cnt;
            d->centroid[0] = v[6] / cnt;
            d->centroid[1] = v[7] / cnt;
            d->centroid[2] = v[16] / cnt;
            double I2[3] = {v[8] - cnt * d->centroid[0] * d->centroid[0],
                            v[9] - cnt * d->centroid[1] * d->centroid[1],
                            v[17] - cnt * d->centroid[2] * d->centroid[2]};
            int hor = vert == 0 ? 1 : 0;
            d->aspect_ratio = I2[vert] > 0 ? std::sqrt(I2[hor] / I2[vert]) : 0.0;
            double rad = D == 2 ? std::sqrt(cnt / M_PI) : std::cbrt(3 * cnt / (4 * M_PI));
            d->Re = 2 * p->rhoB0 * std::fabs(d->U[vert]) * rad / p->muB0;
            // Taylor deformation (L - B)/(L + B) and inclination of the major
            // axis in the x-y plane (2D) or x-z plane (3D: walls at z moving
            // along x), from the principal second moments of the red region
            const double cx = d->centroid[0], cb = D == 2 ? d->centroid[1] : d->centroid[2];
            const double Iaa = v[8] - cnt * cx * cx;
            const double Ibb = (D == 2 ? v[9] : v[17]) - cnt * cb * cb;
            const double Iab = (D == 2 ? v[19] : v[18]) - cnt * cx * cb;
            const double tr = 0.5 * (Iaa + Ibb);
            const double dd = std::sqrt(0.25 * (Iaa - Ibb) * (Iaa - Ibb) + Iab * Iab);
            const double l1 = tr + dd, l2 = tr - dd;
            if (l2 > 0) {
                const double L = std::sqrt(l1), B = std::sqrt(l2);
                d->deformation = (L - B) / (L + B);
            }
            d->inclination = 0.5 * std::atan2(2 * Iab, Iaa - Ibb);
        }
        if (v[11] > 0) {
            d->psi_av = v[10] / v[11];
            d->psi_min = -v[NDIAG + 0];
            d->psi_max = v[NDIAG + 1];
        }
        d->umax = v[NDIAG + 2];
        d->sor_iters_psi = d->sor_iters_C = h.sor_iters;
        d->sor_rounds = h.sor_iters / sweeps_per_round();
        if (h.sor_iters > 0) last_rounds = h.sor_iters / sweeps_per_round();
        d->step = h.step;
        return LBS_OK;
    }
};

int validate(const lbs_params *p, char *err, size_t n) {
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) {
        snprintf(err, n, "grid %dx%dx%d: every size must be positive", p->nx, p->ny, p->nz);
        return LBS_EINVAL;
    }
    if ((long long)p->nx * p->ny * p->nz > (1LL << 31) - 1) {
        snprintf(err, n, "grid %dx%dx%d: more than 2^31 - 1 cells", p->nx, p->ny, p->nz);
        return LBS_EINVAL;
    }
    if (p->nz == 1 && p->wall[2]) {
        snprintf(err, n, "a 2D grid (nz == 1) cannot have walls on z");
        return LBS_EINVAL;
    }
    int dims[3] = {p->nx, p->ny, p->nz};
    for (int a = 0; a < 3; a++) {
        // 3D red-black SOR updates in place: a periodic axis of odd length
        // would make cells of one colour neighbours across the seam
        if (p->nz > 1 && !p->wall[a] && (dims[a] & 1)) {
            snprintf(err, n, "3D grids need an even size on periodic axis %d (got %d)", a, dims[a]);
            return LBS_EINVAL;
        }
        if (p->wall[a] < 0 || p->wall[a] > 2) {
            snprintf(err, n, "axis %d: 0 periodic, 1 bounce-back walls, 2 mirror planes (got %d)",
                     a, p->wall[a]);
            return LBS_EINVAL;
        }
        if (p->wall[a] && dims[a] < 3) {
            snprintf(err, n, "walled axis %d needs at least 3 nodes", a);
            return LBS_EINVAL;
        }
        if (p->wall[a] == 2) {
            for (int b = 0; b < 3; b++)
                if (p->uw_lo[a][b] != 0 || p->uw_hi[a][b] != 0) {
                    snprintf(err, n, "mirror planes do not move (axis %d)", a);
                    return LBS_EINVAL;
                }
        }
        if (p->uw_lo[a][a] != 0 || p->uw_hi[a][a] != 0) {
            snprintf(err, n, "walls move tangentially only (axis %d)", a);
            return LBS_EINVAL;
        }
    }
    if (!(p->rhoR0 > 0 && p->rhoB0 > 0 && p->muR0 > 0 && p->muB0 > 0)) {
        snprintf(err, n, "densities and viscosities must be positive");
        return LBS_EINVAL;
    }
    if (!(p->alphaR < 1 && p->alphaB < 1)) {
        snprintf(err, n, "alpha must be below 1");
        return LBS_EINVAL;
    }
    if (p->sor_max_iter < 1 || p->sor_max_iter > KMAX_SWEEPS) {
        snprintf(err, n, "sor_max_iter must be in [1, %d]", KMAX_SWEEPS);
        return LBS_EINVAL;
    }
    if (!(p->psi_inf > 0) || p->sor_omega <= 0 || p->sor_omega >= 2) {
        snprintf(err, n, "psi_inf > 0 and 0 < omega < 2 required");
        return LBS_EINVAL;
    }
    return LBS_OK;
}

}  // namespace

namespace lbs {

int validate_params(const lbs_params *p, char *err, size_t n) { return validate(p, err, n); }

Base *make_solver(lbs_ctx *ctx) {
    switch (ctx->storage) {
    case LBS_F64: return new (std::nothrow) Solver<double, double>(ctx);
    case LBS_F32: return new (std::nothrow) Solver<float, float>(ctx);
    case LBS_F16: return new (std::nothrow) Solver<float, __half>(ctx);
    case LBS_BF16: return new (std::nothrow) Solver<float, __nv_bfloat16>(ctx);
    }
    return nullptr;
}

}  // namespace lbs

extern "C" {

int lbs_params_default(lbs_params *p, int nx, int ny, int nz) {
    if (!p) return LBS_EINVAL;
    std::memset(p, 0, sizeof(*p));
    p->nx = nx;
    p->ny = ny;
    p->nz = nz;
    p->rhoR0 = p->rhoB0 = 1.0;
    p->muR0 = p->muB0 = 0.1;
    p->alphaR = p->alphaB = nz == 1 ? 4.0 / 9.0 : 1.0 / 3.0;
    p->sigma0 = 0.1;
    p->sigma_min_ratio = 0.1;
    p->E0 = 0.5;
    p->psi_inf = 1.0;
    p->beta = 0.7;
    p->transport = 1;
    p->Ds = p->Db = 0.1;
    p->sor_omega = 1.2;
    p->sor_tol = 5e-7;
    p->sor_max_iter = 40;
    p->eps_w = 1e-6;
    p->eps_n = 1e-6;
    return LBS_OK;
}

size_t lbs_workspace_bytes(const lbs_params *p, int storage) {
    if (!p) return 0;
    char e[256];
    if (validate(p, e, sizeof(e))) return 0;
    switch (storage) {
    case LBS_F64: return layout_of<double, double>(p).total;
    case LBS_F32: return layout_of<float, float>(p).total;
    case LBS_F16: return layout_of<float, __half>(p).total;
    case LBS_BF16: return layout_of<float, __nv_bfloat16>(p).total;
    }
    return 0;
}

int lbs_create(const lbs_params *p, int storage, void *stream, void *workspace,
               size_t workspace_bytes, lbs_ctx **out) {
    if (!p || !out) return LBS_EINVAL;
    *out = nullptr;
    lbs_ctx *ctx = new (std::nothrow) lbs_ctx();
    if (!ctx) return LBS_ENOMEM;
    std::memset(ctx, 0, sizeof(*ctx));
    ctx->p = *p;
    ctx->storage = storage;
    int r = validate(p, ctx->err, sizeof(ctx->err));
    if (!r && storage != LBS_F64 && storage != LBS_F32 && storage != LBS_F16 &&
        storage != LBS_BF16) {
        set_err(ctx, "unsupported storage %d", storage);
        r = LBS_EINVAL;
    }
    if (r) {
        *out = ctx;  // carries the message; lbs_destroy releases it
        return r;
    }
    size_t need = lbs_workspace_bytes(p, storage);
    if (workspace) {
        if (workspace_bytes < need || ((uintptr_t)workspace & 255)) {
            set_err(ctx, "workspace of %zu bytes (need %zu, 256-byte aligned)", workspace_bytes,
                    need);
            *out = ctx;
            return LBS_ENOMEM;
        }
        ctx->ws = workspace;
        ctx->ws_bytes = workspace_bytes;
    } else {
        cudaError_t e = cudaMalloc(&ctx->ws, need);
        if (e != cudaSuccess) {
            set_err(ctx, "cudaMalloc(%zu) failed: %s", need, cudaGetErrorString(e));
            ctx->ws = nullptr;
            *out = ctx;
            return LBS_ENOMEM;
        }
        ctx->own_ws = true;
        ctx->ws_bytes = need;
    }
    if (stream) {
        ctx->stream = (cudaStream_t)stream;
    } else {
        if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
            set_err(ctx, "cudaStreamCreate failed");
            *out = ctx;
            return LBS_ECUDA;
        }
        ctx->own_stream = true;
    }
    ctx->impl = make_solver(ctx);
    *out = ctx;
    if (!ctx->impl) return LBS_ENOMEM;
    return LBS_OK;
}

int lbs_init_fields(lbs_ctx *c, const double *phi, const double *psi, const double *C,
                    const double *u) {
    if (!c || !c->impl || !phi) return LBS_EINVAL;
    return c->impl->init(phi, psi, C, u);
}

int lbs_step(lbs_ctx *c, int n) {
    if (!c || !c->impl || n < 0) return LBS_EINVAL;
    return c->impl->step(n);
}

int lbs_sync(lbs_ctx *c) {
    if (!c || !c->impl) return LBS_EINVAL;
    return c->impl->sync();
}

int lbs_get_fields(lbs_ctx *c, double *rho, double *u, double *phi, double *psi, double *C) {
    if (!c || !c->impl) return LBS_EINVAL;
    return c->impl->get(rho, u, phi, psi, C);
}

int lbs_diagnostics(lbs_ctx *c, lbs_diag *d) {
    if (!c || !c->impl || !d) return LBS_EINVAL;
    return c->impl->diag(d);
}

void lbs_destroy(lbs_ctx *c) {
    if (!c) return;
    if (c->impl) {
        cudaStreamSynchronize(c->stream);
        delete c->impl;
    }
    if (c->own_ws && c->ws) cudaFree(c->ws);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

int lbs_profile(lbs_ctx *c, int enable) {
    if (!c || !c->impl) return LBS_EINVAL;
    return c->impl->profile(enable);
}

int lbs_kernel_times(lbs_ctx *c, double *ms, int n) {
    if (!c || !c->impl || !ms || n < 0) return LBS_EINVAL;
    return c->impl->kernel_times(ms, n);
}

int lbs_get_macro(lbs_ctx *c, double *g, double *a, double *F, double *u, double *S,
                  double *B) {
    if (!c || !c->impl) return LBS_EINVAL;
    return c->impl->macro(g, a, F, u, S, B);
}

int lbs_set_graph(lbs_ctx *c, int enable) {
    if (!c || !c->impl) return LBS_EINVAL;
    return c->impl->set_graph(enable);
}

int lbs_step_result(lbs_ctx *c, double *out) {
    if (!c || !c->impl || !out) return LBS_EINVAL;
    return c->impl->step_result(out);
}

int lbs_set_sor_tile(lbs_ctx *c, int variant) {
    if (!c || !c->impl) return LBS_EINVAL;
    return c->impl->set_sor_tile(variant);
}

int lbs_set_sor_wait_limit(lbs_ctx *c, long long polls) {
    if (!c || !c->impl) return LBS_EINVAL;
    return c->impl->set_sor_wait_limit(polls);
}

int lbs_set_sor_persistent(lbs_ctx *c, int on) {
    if (!c || !c->impl) return LBS_EINVAL;
    return c->impl->set_sor_persistent(on);
}

int lbs_save_state(lbs_ctx *c, void *buf, size_t *bytes) {
    if (!c || !c->impl || !bytes) return LBS_EINVAL;
    return c->impl->save_state(buf, bytes);
}

int lbs_load_state(lbs_ctx *c, const void *buf, size_t bytes) {
    if (!c || !c->impl || !buf) return LBS_EINVAL;
    return c->impl->load_state(buf, bytes);
}

int lbs_step_kernel_count(const lbs_ctx *c) {
    if (!c || !c->impl) return 0;
    return c->impl->kernel_count();
}

const char *lbs_last_error(const lbs_ctx *c) {
    if (!c) return "null context";
    return c->err[0] ? c->err : "no error";
}

}  // extern "C"
