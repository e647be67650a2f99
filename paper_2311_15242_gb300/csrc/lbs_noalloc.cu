// lbs_noalloc.cu — the total surfactant of caller-owned device fields,
// computed without allocating any device memory.
//
// Some callers cannot call cudaMalloc: code that runs where the device's
// memory is owned by another allocator (a framework pool that must not be
// bypassed, or a process that reserved the device memory up front), and
// monitoring loops that must not stall the solver's stream with the implicit
// device synchronisation of an allocation.  For them this entry point keeps
// its scratch (the per-block partial sums and the arrival counter) in a
// file-scope device array of fixed size, which every GPU that loads the
// library holds until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/lbs.h"

namespace {

constexpr int kThreadsX = 32, kThreadsY = 8, kThreads = kThreadsX * kThreadsY;
constexpr int kStrip = 16;                        // cells per thread along y
constexpr int kMaxBlocks = 8192;                  // partial sums held in the scratch
constexpr int kMaxDevices = 64;

// the scratch: 8192 FP64 partials (64 KiB) and one arrival counter
static __device__ __align__(256) double g_scratch_partials[kMaxBlocks];
static __device__ __align__(256) unsigned int g_scratch_ticket;

std::mutex g_setup_mu;
void *g_partials_addr[kMaxDevices];
void *g_ticket_addr[kMaxDevices];

// sum (a + eps) psi + (chi + eps) C: every thread adds a strip of cells with
// a compensated sum in R, strips are added in FP64, the last block to arrive
// adds the block partials in block order and writes the total
template <typename R>
__global__ void k_total_static(const R *a, const R *chi, const R *psi, const R *C, int nx,
                               int rows, long long pitch, R eps_w, double *partials,
                               unsigned int *ticket, double *total) {
    const int x = blockIdx.x * kThreadsX + threadIdx.x;
    const int r0 = (blockIdx.y * kThreadsY + threadIdx.y) * kStrip;
    const int t = threadIdx.y * kThreadsX + threadIdx.x;
    R sum = R(0), comp = R(0);
    if (x < nx)
        for (int k = 0; k < kStrip; k++) {
            const int r = r0 + k;
            if (r >= rows) break;
            const long long c = (long long)r * pitch + x;
            const R v = (a[c] + eps_w) * psi[c] + (chi[c] + eps_w) * C[c];
            const R yv = v - comp;
            const R tt = sum + yv;
            comp = (tt - sum) - yv;
            sum = tt;
        }
    double v = double(sum) - double(comp);
    __shared__ double warp_sums[kThreads / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((t & 31) == 0) warp_sums[t >> 5] = v;
    __syncthreads();
    const unsigned int nblocks = gridDim.x * gridDim.y;
    const unsigned int b = blockIdx.y * gridDim.x + blockIdx.x;
    __shared__ bool last;
    if (t == 0) {
        double s = 0;
        for (int w = 0; w < kThreads / 32; w++) s += warp_sums[w];
        partials[b] = s;
        __threadfence();
        last = atomicAdd(ticket, 1u) == nblocks - 1;
    }
    __syncthreads();
    if (!last) return;
    // the last block: thread t adds partials t, t + kThreads, ... in order
    double s = 0;
    for (unsigned int k = t; k < nblocks; k += kThreads) s += __ldcg(&partials[k]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    __syncthreads();
    if ((t & 31) == 0) warp_sums[t >> 5] = s;
    __syncthreads();
    if (t == 0) {
        double tot = 0;
        for (int w = 0; w < kThreads / 32; w++) tot += warp_sums[w];
        *total = tot;
        *ticket = 0;
    }
}

// device addresses of the scratch for the current device; the first call on
// a device looks them up
int scratch_addresses(void **partials, void **ticket) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LBS_ECUDA;
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_partials_addr[dev]) {
        void *p = nullptr, *q = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch_partials) != cudaSuccess) return LBS_ECUDA;
        if (cudaGetSymbolAddress(&q, g_scratch_ticket) != cudaSuccess) return LBS_ECUDA;
        g_partials_addr[dev] = p;
        g_ticket_addr[dev] = q;
    }
    *partials = g_partials_addr[dev];
    *ticket = g_ticket_addr[dev];
    return LBS_OK;
}

}  // namespace

extern "C" int lbs_surfactant_total_static(int storage, const void *a, const void *chi,
                                           const void *psi, const void *C, int nx, int ny,
                                           int nz, int pitch, double eps_w, double *total,
                                           void *stream) {
    if ((storage != LBS_F32 && storage != LBS_F64) || !a || !chi || !psi || !C || !total)
        return LBS_EINVAL;
    if (nx < 1 || ny < 1 || nz < 1 || pitch < nx) return LBS_EINVAL;
    const long long rows = (long long)ny * nz;
    const long long gx = (nx + kThreadsX - 1) / kThreadsX;
    const long long gy = (rows + (long long)kThreadsY * kStrip - 1) / ((long long)kThreadsY * kStrip);
    // the fixed scratch holds one partial per block: larger grids are refused
    if ((long long)nx * rows > LBS_STATIC_MAX_CELLS || gx * gy > kMaxBlocks || gy > 65535)
        return LBS_EINVAL;
    void *partials = nullptr, *ticket = nullptr;
    int r = scratch_addresses(&partials, &ticket);
    if (r) return r;
    cudaStream_t s = (cudaStream_t)stream;
    // the counter must start at zero whatever an earlier, interrupted call left
    if (cudaMemsetAsync(ticket, 0, sizeof(unsigned int), s) != cudaSuccess) return LBS_ECUDA;
    dim3 grid((unsigned)gx, (unsigned)gy), block(kThreadsX, kThreadsY);
    if (storage == LBS_F32)
        k_total_static<float><<<grid, block, 0, s>>>(
            (const float *)a, (const float *)chi, (const float *)psi, (const float *)C, nx,
            (int)rows, pitch, float(eps_w), (double *)partials, (unsigned int *)ticket, total);
    else
        k_total_static<double><<<grid, block, 0, s>>>(
            (const double *)a, (const double *)chi, (const double *)psi, (const double *)C, nx,
            (int)rows, pitch, eps_w, (double *)partials, (unsigned int *)ticket, total);
    return cudaGetLastError() == cudaSuccess ? LBS_OK : LBS_ECUDA;
}
