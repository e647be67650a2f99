// lbs_batch.cu — a batch of independent 2D instances (a parameter sweep of
// the coupled step: different grids, Eotvos and Biot numbers, confinement)
// advanced together.
//
// Every phase of the step is one launch for the whole batch: a grid of
// (SM count x resident blocks) blocks walks a work list of (instance, tile)
// items, copies the instance's descriptor into shared memory when the
// instance changes and runs the same per-cell bodies as the single-instance
// kernels.  The SOR rounds of all instances share one WHILE node: each
// instance keeps its own round counter, convergence test and ping-pong
// parity, a converged instance's tiles skip the remaining rounds, and the
// loop ends when no instance is still iterating.  A CUDA graph holds several
// whole steps.  The cell-tile shape (block shape) and the SOR tile are
// chosen at run time (lbs_batch_set_tiles; the autotuner picks them).
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "lbs_internal.h"
#include "lbs_k2d.cuh"

using namespace lbs;

namespace {

struct WorkItem {
    int inst, x0, y0, a0, a1, pad[3];  // 32 bytes
};

struct BatchCtl {
    unsigned int ticket;  // arrival counter of the SOR launch's blocks
    int active;           // instances still iterating in the current solve
};

enum { OP_FORCE, OP_FDCOLLIDE, OP_STREAM, OP_GRAD, OP_SCALE, NOPS };

// copy descriptor k into shared memory (all threads; uniform) and return
// whether the instance is alive (an instance whose total went non-finite is
// skipped from then on; the flag is read once per change of instance)
template <typename R>
__device__ __forceinline__ bool load_inst(const Inst<R> *insts, int k, Inst<R> &sI, int &cur,
                                          int &alive) {
    if (k == cur) return alive;
    __syncthreads();
    const int n = (int)(sizeof(Inst<R>) / 4);
    const int *src = (const int *)(insts + k);
    int *dst = (int *)&sI;
    const int nt = blockDim.x * blockDim.y;
    for (int i = threadIdx.x + threadIdx.y * blockDim.x; i < n; i += nt) dst[i] = src[i];
    __shared__ int s_alive;
    if (threadIdx.x == 0 && threadIdx.y == 0) s_alive = !insts[k].ctl->dead;
    __syncthreads();
    cur = k;
    alive = s_alive;
    return alive;
}

// one per-cell phase over the batch; work item = tile origin (x0, y0) of
// blockDim.x x blockDim.y cells of instance `inst`
template <typename R, typename P, int OP>
__global__ void kb_cells2(const Inst<R> *__restrict__ insts, const WorkItem *__restrict__ work,
                          int nwork) {
    __shared__ Inst<R> sI;
    int cur = -1, alive = 0;
    for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
        const WorkItem it = work[w];
        if (!load_inst(insts, it.inst, sI, cur, alive)) continue;
        const int x = it.x0 + threadIdx.x, y = it.y0 + threadIdx.y;
        if (OP == OP_FORCE)
            force2_cell(sI, x, y);
        else if (OP == OP_FDCOLLIDE) {
            // (the explicit surfactant terms and the collision in one pass)
            fd2_cell(sI, x, y, nullptr, nullptr);
            collide2_cell<R, P>(sI, x, y);
        }
        else if (OP == OP_STREAM)
            stream2_cell<R, P>(sI, x, y);
        else if (OP == OP_GRAD)
            grad2_cell(sI, x, y);
        else
            scale2_cell(sI, x, y, 0);
    }
}

// opens the SOR solve of every live instance in the work lists (act[k])
template <typename R>
__global__ void kb_sor_begin(const Inst<R> *insts, const int *act, int n, BatchCtl *bc) {
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        Ctl *ctl = insts[k].ctl;
        const int a = act[k] && !ctl->dead;
        ctl->sor_active = a;
        if (a) atomicAdd(&cnt, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        bc->active = cnt;
        bc->ticket = 0;
    }
}

// one blocked SOR round of every instance still iterating; work item =
// SOR tile (x0, y0) = (bx, by) of instance `inst`, a0 = its tile count.
// graph: 1 inside the WHILE node (the last block ends the loop when no
// instance is active), 0 for a host-driven loop (reads bc->active)
template <typename R, int TX, int TY, int K, int BS>
__global__ void __launch_bounds__(BS)
    kb_sor2(const Inst<R> *__restrict__ insts, const WorkItem *__restrict__ work, int nwork,
            BatchCtl *bc, cudaGraphConditionalHandle loop, int max_rounds, int graph) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Inst<R> sI;
    __shared__ int s_round;
    int cur = -1, alive = 0;
    const int tid = threadIdx.x;
    for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
        const WorkItem it = work[w];
        load_inst(insts, it.inst, sI, cur, alive);
        __syncthreads();
        if (tid == 0) s_round = sI.ctl->sor_active ? sI.ctl->sor_exec : -1;
        __syncthreads();
        const int round = s_round;
        if (round < 0) continue;  // converged earlier in this solve
        sor_tile2<R, TX, TY, K, BS>(sI, round, it.x0, it.y0, smem_raw);
        if (last_block(&sI.ctl->sor_ticket, (unsigned)it.a0) && tid == 0) {
            Ctl *ctl = sI.ctl;
            ctl->sor_ticket = 0;
            const bool stop = sor_round_stop<R>(ctl, round, double(sI.sor_tol), max_rounds);
            ctl->sor_exec = round + 1;
            if (stop) {
                ctl->sor_active = 0;
                atomicSub(&bc->active, 1);
            }
        }
    }
    if (last_block(&bc->ticket, gridDim.x) && tid == 0) {
        bc->ticket = 0;
        if (graph && atomicAdd(&bc->active, 0) <= 0) cudaGraphSetConditional(loop, 0);
    }
}

// total surfactant and rescale factor of every instance (end of step);
// work item = block (x0, y0) = (bx, by) of the instance's strip grid,
// a0 = its block count, a1 = its grid width
template <typename R, int BS>
__global__ void kb_surf2(const Inst<R> *__restrict__ insts, const WorkItem *__restrict__ work,
                         int nwork, int sweeps_per_round) {
    __shared__ Inst<R> sI;
    int cur = -1, alive = 0;
    for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
        const WorkItem it = work[w];
        if (!load_inst(insts, it.inst, sI, cur, alive)) continue;
        surf2_block<R, BS>(sI, 1, it.a0, sweeps_per_round, it.x0, it.y0, it.a1);
        __syncthreads();
    }
}

constexpr int kSurfBX = 32, kSurfBY = 8, kSurfBS = kSurfBX * kSurfBY;

#define LBS_SORV(v) sor_vtx(v), sor_vty(v), sor_vk(v), sor_vbs(v)
template <typename R>
void *sor_kernel_t(int v) {
    switch (v) {
    case 1: return (void *)kb_sor2<R, LBS_SORV(1)>;
    case 2: return (void *)kb_sor2<R, LBS_SORV(2)>;
    case 3: return (void *)kb_sor2<R, LBS_SORV(3)>;
    case 4: return (void *)kb_sor2<R, LBS_SORV(4)>;
    case 5: return (void *)kb_sor2<R, LBS_SORV(5)>;
    case 6: return (void *)kb_sor2<R, LBS_SORV(6)>;
    case 7: return (void *)kb_sor2<R, LBS_SORV(7)>;
    case 8: return (void *)kb_sor2<R, LBS_SORV(8)>;
    default: return (void *)kb_sor2<R, LBS_SORV(0)>;
    }
}
void *sor_kernel(bool dbl, int v) { return dbl ? sor_kernel_t<double>(v) : sor_kernel_t<float>(v); }

template <typename R>
size_t sor_smem(int v) {
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
void sor_tile_shape(int v, int &tx, int &ty) {
    tx = sor_vtx(v);
    ty = sor_vty(v);
}

}  // namespace

struct lbs_batch {
    virtual ~lbs_batch() {}
    virtual int init(int k, const double *, const double *, const double *, const double *) = 0;
    virtual int set_tiles(int tx, int ty, int sor_variant) = 0;
    virtual int step(int n) = 0;
    virtual int sync() = 0;
    virtual int get(int k, double *, double *, double *, double *, double *) = 0;
    virtual int diag(lbs_diag *) = 0;
    virtual int kernel_count() const = 0;
    virtual int set_graph(int on) = 0;
    virtual int status(int *st) = 0;
    virtual int set_active(int k, int on) = 0;
    char err[512] = {0};
};

namespace {

void berr(lbs_batch *b, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(b->err, sizeof(b->err), fmt, ap);
    va_end(ap);
}

#define BCK(call)                                                                          \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            berr(this, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__,   \
                 __LINE__);                                                                \
            return LBS_ECUDA;                                                              \
        }                                                                                  \
    } while (0)

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

template <typename R, typename P>
struct Batch : lbs_batch {
    int n = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    void *ws = nullptr;
    bool own_ws = false;
    std::vector<lbs_ctx *> ctxs;
    Inst<R> *d_insts = nullptr;
    BatchCtl *d_bc = nullptr;
    int *d_act = nullptr;      // instance in the work lists (device copy of act)
    std::vector<int> act;      // host flags: instance in the work lists
    std::vector<int> st;       // sticky per-instance status (lbs_status codes)
    WorkItem *d_cells = nullptr, *d_sor = nullptr, *d_surf = nullptr;
    int n_cells = 0, n_sor = 0, n_surf = 0;
    int tx = 32, ty = 8, sv = 0;
    int g_cells[NOPS] = {0}, g_sor = 0, g_surf = 0;
    int max_rounds = 1;
    int max_iter = 1;  // largest sor_max_iter of the instances
    int last_rounds = 4;
    bool use_graph = true;
    static constexpr int kGraphSteps = 8;
    cudaGraph_t graph[2] = {nullptr, nullptr};
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};

    ~Batch() override {
        if (stream) cudaStreamSynchronize(stream);
        drop_graphs();
        for (auto *c : ctxs) {
            if (c->impl) delete c->impl;
            delete c;
        }
        cudaFree(d_insts);
        cudaFree(d_bc);
        cudaFree(d_act);
        cudaFree(d_cells);
        cudaFree(d_sor);
        cudaFree(d_surf);
        if (own_ws && ws) cudaFree(ws);
        if (own_stream && stream) cudaStreamDestroy(stream);
    }

    void drop_graphs() {
        for (int k = 0; k < 2; k++) {
            if (gexec[k]) cudaGraphExecDestroy(gexec[k]);
            if (graph[k]) cudaGraphDestroy(graph[k]);
            gexec[k] = nullptr;
            graph[k] = nullptr;
        }
    }

    int create(const lbs_params *p, int nn, int storage, void *strm, void *workspace,
               size_t bytes) {
        n = nn;
        if (strm) {
            stream = (cudaStream_t)strm;
        } else {
            BCK(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking));
            own_stream = true;
        }
        std::vector<size_t> off(n);
        size_t total = 0;
        for (int k = 0; k < n; k++) {
            off[k] = total;
            total = align256(total + lbs_workspace_bytes(&p[k], storage));
        }
        if (workspace) {
            if (bytes < total || ((uintptr_t)workspace & 255)) {
                berr(this, "workspace of %zu bytes (need %zu, 256-byte aligned)", bytes, total);
                return LBS_ENOMEM;
            }
            ws = workspace;
        } else {
            BCK(cudaMalloc(&ws, total));
            own_ws = true;
        }
        std::vector<Inst<R>> h(n);
        for (int k = 0; k < n; k++) {
            lbs_ctx *c = new (std::nothrow) lbs_ctx();
            if (!c) return LBS_ENOMEM;
            std::memset(c, 0, sizeof(*c));
            ctxs.push_back(c);
            c->p = p[k];
            c->storage = storage;
            c->stream = stream;
            c->ws = (char *)ws + off[k];
            c->ws_bytes = lbs_workspace_bytes(&p[k], storage);
            c->impl = make_solver(c);
            if (!c->impl) return LBS_ENOMEM;
            if (c->impl->inst_bytes() != sizeof(Inst<R>)) {
                berr(this, "internal: descriptor size mismatch");
                return LBS_EINVAL;
            }
            // the batch runs the separate per-cell kernels: populations and
            // moments return to set 0 every step and the SOR starting guess
            // sits in psi, C
            c->impl->set_batch_member();
            std::memcpy(&h[k], c->impl->inst(), sizeof(Inst<R>));
            if (p[k].sor_max_iter > max_iter) max_iter = p[k].sor_max_iter;
        }
        BCK(cudaMalloc(&d_insts, n * sizeof(Inst<R>)));
        BCK(cudaMemcpy(d_insts, h.data(), n * sizeof(Inst<R>), cudaMemcpyHostToDevice));
        BCK(cudaMalloc(&d_bc, sizeof(BatchCtl)));
        BCK(cudaMemset(d_bc, 0, sizeof(BatchCtl)));
        act.assign(n, 1);
        st.assign(n, 0);
        BCK(cudaMalloc(&d_act, n * sizeof(int)));
        BCK(cudaMemcpy(d_act, act.data(), n * sizeof(int), cudaMemcpyHostToDevice));
        for (int v = 0; v < kSorVariants; v++) {
            if (!sor_fits(v)) continue;
            void *f = sor_kernel(sizeof(R) == 8, v);
            BCK(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)sor_smem<R>(v)));
        }
        return set_tiles(32, 8, 0);
    }

    // resident blocks of kernel f x SM count (a persistent grid), capped by the work
    int persistent_grid(const void *f, int threads, size_t smem, int nwork) {
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, f, threads, smem);
        if (per < 1) per = 1;
        long long g = (long long)sms * per;
        if (g > nwork) g = nwork;
        return g < 1 ? 1 : (int)g;
    }

    int upload(WorkItem *&d, const std::vector<WorkItem> &h) {
        if (d) cudaFree(d);
        d = nullptr;
        if (h.empty()) return LBS_OK;
        BCK(cudaMalloc(&d, h.size() * sizeof(WorkItem)));
        BCK(cudaMemcpy(d, h.data(), h.size() * sizeof(WorkItem), cudaMemcpyHostToDevice));
        return LBS_OK;
    }

    static bool sor_fits(int v) {
        int dev = 0, lim = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&lim, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        return sor_smem<R>(v) <= (size_t)lim;
    }

    int set_tiles(int tx_, int ty_, int sv_) override {
        if (tx_ < 1 || ty_ < 1 || tx_ * ty_ > 1024 || (tx_ * ty_) % 32 || sv_ < 0 ||
            sv_ >= kSorVariants) {
            berr(this, "tile %dx%d / SOR variant %d: block of 32..1024 threads (a multiple of 32) "
                       "and variant 0..%d required", tx_, ty_, sv_, kSorVariants - 1);
            return LBS_EINVAL;
        }
        if (!sor_fits(sv_)) {
            berr(this, "SOR variant %d needs %zu bytes of shared memory a block in this storage "
                       "form", sv_, sor_smem<R>(sv_));
            return LBS_EINVAL;
        }
        BCK(cudaStreamSynchronize(stream));
        drop_graphs();
        tx = tx_;
        ty = ty_;
        sv = sv_;
        max_rounds = (max_iter + sor_vk(sv) - 1) / sor_vk(sv);
        int stx, sty;
        sor_tile_shape(sv, stx, sty);
        std::vector<WorkItem> cells, sor, surf;
        for (int k = 0; k < n; k++) {
            if (!act[k]) continue;
            const lbs_params &p = ctxs[k]->p;
            for (int y0 = 0; y0 < p.ny; y0 += ty)
                for (int x0 = 0; x0 < p.nx; x0 += tx) cells.push_back({k, x0, y0, 0, 0, {0, 0, 0}});
            const int sx = (p.nx + stx - 1) / stx, sy = (p.ny + sty - 1) / sty;
            for (int by = 0; by < sy; by++)
                for (int bx = 0; bx < sx; bx++) sor.push_back({k, bx, by, sx * sy, 0, {0, 0, 0}});
            const int gx = (p.nx + kSurfBX - 1) / kSurfBX;
            const int gy = (p.ny + kSurfBY * SURF_STRIP - 1) / (kSurfBY * SURF_STRIP);
            for (int by = 0; by < gy; by++)
                for (int bx = 0; bx < gx; bx++) surf.push_back({k, bx, by, gx * gy, gx, {0, 0, 0}});
        }
        int r;
        if ((r = upload(d_cells, cells)) || (r = upload(d_sor, sor)) || (r = upload(d_surf, surf)))
            return r;
        n_cells = (int)cells.size();
        n_sor = (int)sor.size();
        n_surf = (int)surf.size();
        BCK(cudaMemcpy(d_act, act.data(), n * sizeof(int), cudaMemcpyHostToDevice));
        const int th = tx * ty;
        const void *fk[NOPS] = {(void *)kb_cells2<R, P, OP_FORCE>, (void *)kb_cells2<R, P, OP_FDCOLLIDE>,
                             (void *)kb_cells2<R, P, OP_STREAM>, (void *)kb_cells2<R, P, OP_GRAD>,
                             (void *)kb_cells2<R, P, OP_SCALE>};
        for (int o = 0; o < NOPS; o++) g_cells[o] = persistent_grid(fk[o], th, 0, n_cells);
        g_sor = persistent_grid(sor_kernel(sizeof(R) == 8, sv), sor_vbs(sv), sor_smem<R>(sv), n_sor);
        g_surf = persistent_grid((void *)kb_surf2<R, kSurfBS>, kSurfBS, 0, n_surf);
        return LBS_OK;
    }

    int init(int k, const double *phi, const double *psi, const double *C,
             const double *u) override {
        if (k < 0 || k >= n) {
            berr(this, "instance %d of %d", k, n);
            return LBS_EINVAL;
        }
        int r = ctxs[k]->impl->init(phi, psi, C, u);
        if (r) berr(this, "instance %d: %s", k, ctxs[k]->err);
        return r;
    }

    // the launches of one step of the whole batch
    int enqueue_step(cudaStream_t s, bool capturing) {
        const dim3 blk(tx, ty, 1);
        kb_cells2<R, P, OP_FORCE><<<g_cells[OP_FORCE], blk, 0, s>>>(d_insts, d_cells, n_cells);
        kb_cells2<R, P, OP_FDCOLLIDE><<<g_cells[OP_FDCOLLIDE], blk, 0, s>>>(d_insts, d_cells,
                                                                          n_cells);
        kb_cells2<R, P, OP_STREAM><<<g_cells[OP_STREAM], blk, 0, s>>>(d_insts, d_cells, n_cells);
        kb_cells2<R, P, OP_GRAD><<<g_cells[OP_GRAD], blk, 0, s>>>(d_insts, d_cells, n_cells);
        kb_sor_begin<R><<<1, 256, 0, s>>>(d_insts, d_act, n, d_bc);
        void *fsor = sor_kernel(sizeof(R) == 8, sv);
        const size_t smem = sor_smem<R>(sv);
        if (capturing) {
            cudaStreamCaptureStatus st;
            cudaGraph_t cg;
            const cudaGraphNode_t *deps = nullptr;
            size_t nd = 0;
            BCK(cudaStreamGetCaptureInfo(s, &st, nullptr, &cg, &deps, nullptr, &nd));
            cudaGraphConditionalHandle h;
            BCK(cudaGraphConditionalHandleCreate(&h, cg, 1, cudaGraphCondAssignDefault));
            cudaGraphNodeParams cp = {};
            cp.type = cudaGraphNodeTypeConditional;
            cp.conditional.handle = h;
            cp.conditional.type = cudaGraphCondTypeWhile;
            cp.conditional.size = 1;
            cudaGraphNode_t cnode;
            BCK(cudaGraphAddNode(&cnode, cg, deps, nullptr, nd, &cp));
            int graph_mode = 1;
            void *args[] = {(void *)&d_insts, (void *)&d_sor, (void *)&n_sor, (void *)&d_bc,
                            (void *)&h, (void *)&max_rounds, (void *)&graph_mode};
            cudaKernelNodeParams kp = {};
            kp.func = fsor;
            kp.gridDim = dim3(g_sor, 1, 1);
            kp.blockDim = dim3(sor_vbs(sv), 1, 1);
            kp.sharedMemBytes = (unsigned)smem;
            kp.kernelParams = args;
            cudaGraphNode_t kn;
            BCK(cudaGraphAddKernelNode(&kn, cp.conditional.phGraph_out[0], nullptr, 0, &kp));
            BCK(cudaStreamUpdateCaptureDependencies(s, &cnode, nullptr, 1,
                                                    cudaStreamSetCaptureDependencies));
        } else {
            // host-driven rounds (for profilers): stop when no instance is active
            cudaGraphConditionalHandle h0 = 0;
            int graph_mode = 0;
            for (int r = 0; r < max_rounds; r++) {
                void *args[] = {(void *)&d_insts, (void *)&d_sor, (void *)&n_sor, (void *)&d_bc,
                                (void *)&h0, (void *)&max_rounds, (void *)&graph_mode};
                BCK(cudaLaunchKernel(fsor, dim3(g_sor), dim3(sor_vbs(sv)), args, smem, s));
                BatchCtl hb;
                BCK(cudaMemcpyAsync(&hb, d_bc, sizeof(hb), cudaMemcpyDeviceToHost, s));
                BCK(cudaStreamSynchronize(s));
                if (hb.active <= 0) break;
            }
        }
        kb_surf2<R, kSurfBS><<<g_surf, dim3(kSurfBX, kSurfBY), 0, s>>>(d_insts, d_surf, n_surf,
                                                                       sor_vk(sv));
        kb_cells2<R, P, OP_SCALE><<<g_cells[OP_SCALE], blk, 0, s>>>(d_insts, d_cells, n_cells);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            berr(this, "kernel launch failed: %s", cudaGetErrorString(e));
            return LBS_ECUDA;
        }
        return LBS_OK;
    }

    int build(int which, int steps) {
        BCK(cudaGraphCreate(&graph[which], 0));
        BCK(cudaStreamBeginCaptureToGraph(stream, graph[which], nullptr, nullptr, 0,
                                          cudaStreamCaptureModeThreadLocal));
        int r = LBS_OK;
        for (int k = 0; k < steps && !r; k++) r = enqueue_step(stream, true);
        cudaGraph_t out = nullptr;
        cudaError_t e = cudaStreamEndCapture(stream, &out);
        if (r) return r;
        if (e != cudaSuccess) {
            berr(this, "graph capture failed: %s", cudaGetErrorString(e));
            return LBS_ECUDA;
        }
        BCK(cudaGraphInstantiate(&gexec[which], graph[which], 0));
        return LBS_OK;
    }

    int step(int nsteps) override {
        if (nsteps <= 0) return LBS_OK;
        if (!use_graph) {
            for (int k = 0; k < nsteps; k++) {
                int r = enqueue_step(stream, false);
                if (r) return r;
            }
            return LBS_OK;
        }
        // graph 0: kGraphSteps steps; graph 1: one step (the remainder)
        const int big = nsteps / kGraphSteps, rest = nsteps % kGraphSteps;
        if (big && !gexec[0]) {
            int r = build(0, kGraphSteps);
            if (r) return r;
        }
        if (rest && !gexec[1]) {
            int r = build(1, 1);
            if (r) return r;
        }
        for (int k = 0; k < big; k++) BCK(cudaGraphLaunch(gexec[0], stream));
        for (int k = 0; k < rest; k++) BCK(cudaGraphLaunch(gexec[1], stream));
        return LBS_OK;
    }

    // reads (and clears on the device) every instance's status into the
    // sticky host copy; CUDA failures are returned
    int collect() {
        BCK(cudaStreamSynchronize(stream));
        for (int k = 0; k < n; k++) {
            int r = ctxs[k]->impl->sync();
            if (r == LBS_ECUDA) {
                berr(this, "instance %d: %s", k, ctxs[k]->err);
                return r;
            }
            if (r && !st[k]) st[k] = r;
        }
        return LBS_OK;
    }

    // fails with the first instance (in the work lists) whose solve failed
    int sync() override {
        int r = collect();
        if (r) return r;
        for (int k = 0; k < n; k++)
            if (act[k] && st[k]) {
                berr(this, "instance %d: %s", k, ctxs[k]->err);
                return st[k];
            }
        return LBS_OK;
    }

    int status(int *out) override {
        int r = collect();
        if (r) return r;
        for (int k = 0; k < n; k++) {
            out[k] = st[k];
            st[k] = 0;
        }
        return LBS_OK;
    }

    int set_active(int k, int on) override {
        if (k < 0 || k >= n) {
            berr(this, "instance %d of %d", k, n);
            return LBS_EINVAL;
        }
        if (act[k] == (on ? 1 : 0)) return LBS_OK;
        act[k] = on ? 1 : 0;
        return set_tiles(tx, ty, sv);
    }

    int get(int k, double *rho, double *u, double *phi, double *psi, double *C) override {
        if (k < 0 || k >= n) {
            berr(this, "instance %d of %d", k, n);
            return LBS_EINVAL;
        }
        int r = collect();
        if (r) return r;
        r = ctxs[k]->impl->get(rho, u, phi, psi, C);
        if (r) berr(this, "instance %d: %s", k, ctxs[k]->err);
        return r;
    }

    // diagnostics of every instance; failed solves are reported through
    // lbs_batch_status, not here
    int diag(lbs_diag *d) override {
        int r = collect();
        if (r) return r;
        int rounds = 0;
        for (int k = 0; k < n; k++) {
            r = ctxs[k]->impl->diag(&d[k]);
            if (r) {
                berr(this, "instance %d: %s", k, ctxs[k]->err);
                return r;
            }
            if (d[k].sor_rounds > rounds) rounds = d[k].sor_rounds;
        }
        if (rounds > 0) last_rounds = rounds;
        return LBS_OK;
    }

    // launches of one step: 4 cell phases (fd fused with collide), the SOR
    // opener, the rounds of the slowest instance at the last diagnostics, the
    // total and the rescale
    int kernel_count() const override { return 7 + last_rounds; }

    int set_graph(int on) override {
        use_graph = bool(on);
        return LBS_OK;
    }
};

int check_batch(const lbs_params *p, int n, int storage, char *err, size_t len) {
    if (!p || n < 1) {
        snprintf(err, len, "a batch needs at least one instance");
        return LBS_EINVAL;
    }
    if (storage != LBS_F64 && storage != LBS_F32 && storage != LBS_F16 && storage != LBS_BF16) {
        snprintf(err, len, "unsupported storage %d", storage);
        return LBS_EINVAL;
    }
    for (int k = 0; k < n; k++) {
        char e[256];
        if (validate_params(&p[k], e, sizeof(e))) {
            snprintf(err, len, "instance %d: %s", k, e);
            return LBS_EINVAL;
        }
        if (p[k].nz != 1 || !p[k].transport) {
            snprintf(err, len, "instance %d: batches hold 2D instances with surfactant transport", k);
            return LBS_EINVAL;
        }
    }
    return LBS_OK;
}

}  // namespace

extern "C" {

size_t lbs_batch_workspace_bytes(const lbs_params *p, int n, int storage) {
    char e[256];
    if (check_batch(p, n, storage, e, sizeof(e))) return 0;
    size_t total = 0;
    for (int k = 0; k < n; k++) total = align256(total + lbs_workspace_bytes(&p[k], storage));
    return total;
}

int lbs_batch_create(const lbs_params *p, int n, int storage, void *stream, void *workspace,
                     size_t workspace_bytes, lbs_batch **out) {
    if (!out) return LBS_EINVAL;
    *out = nullptr;
    lbs_batch *b = nullptr;
    switch (storage) {
    case LBS_F64: b = new (std::nothrow) Batch<double, double>(); break;
    case LBS_F32: b = new (std::nothrow) Batch<float, float>(); break;
    case LBS_F16: b = new (std::nothrow) Batch<float, __half>(); break;
    default: b = new (std::nothrow) Batch<float, __nv_bfloat16>(); break;
    }
    if (!b) return LBS_ENOMEM;
    *out = b;
    int r = check_batch(p, n, storage, b->err, sizeof(b->err));
    if (r) return r;
    switch (storage) {
    case LBS_F64: return ((Batch<double, double> *)b)->create(p, n, storage, stream, workspace, workspace_bytes);
    case LBS_F32: return ((Batch<float, float> *)b)->create(p, n, storage, stream, workspace, workspace_bytes);
    case LBS_F16: return ((Batch<float, __half> *)b)->create(p, n, storage, stream, workspace, workspace_bytes);
    default: return ((Batch<float, __nv_bfloat16> *)b)->create(p, n, storage, stream, workspace, workspace_bytes);
    }
}

int lbs_batch_init_fields(lbs_batch *b, int k, const double *phi, const double *psi,
                          const double *C, const double *u) {
    if (!b || !phi) return LBS_EINVAL;
    return b->init(k, phi, psi, C, u);
}

int lbs_batch_set_tiles(lbs_batch *b, int tx, int ty, int sor_tile) {
    if (!b) return LBS_EINVAL;
    return b->set_tiles(tx, ty, sor_tile);
}

int lbs_batch_step(lbs_batch *b, int n) {
    if (!b || n < 0) return LBS_EINVAL;
    return b->step(n);
}

int lbs_batch_sync(lbs_batch *b) {
    if (!b) return LBS_EINVAL;
    return b->sync();
}

int lbs_batch_get_fields(lbs_batch *b, int k, double *rho, double *u, double *phi, double *psi,
                         double *C) {
    if (!b) return LBS_EINVAL;
    return b->get(k, rho, u, phi, psi, C);
}

int lbs_batch_diagnostics(lbs_batch *b, lbs_diag *d) {
    if (!b || !d) return LBS_EINVAL;
    return b->diag(d);
}

int lbs_batch_set_graph(lbs_batch *b, int enable) {
    if (!b) return LBS_EINVAL;
    return b->set_graph(enable);
}

int lbs_batch_step_kernel_count(const lbs_batch *b) { return b ? b->kernel_count() : 0; }

int lbs_batch_status(lbs_batch *b, int *status) {
    if (!b || !status) return LBS_EINVAL;
    return b->status(status);
}

int lbs_batch_set_active(lbs_batch *b, int k, int active) {
    if (!b) return LBS_EINVAL;
    return b->set_active(k, active);
}

void lbs_batch_destroy(lbs_batch *b) {
    if (!b) return;
    delete b;
}

const char *lbs_batch_last_error(const lbs_batch *b) {
    if (!b) return "null batch";
    return b->err[0] ? b->err : "no error";
}

}  // extern "C"
