// lbs_launch3.h — host-side launchers of the D3Q19 kernels.  The kernels are
// instantiated in their own translation unit (lbs_3d.cu) so that the D2Q9
// and D3Q19 code compile in parallel.
#pragma once

#include <cuda_runtime.h>

#include "lbs_dev.cuh"

namespace lbs {

template <typename R, typename P>
struct Launch3 {
    static void init(const Inst<R> &I, dim3 g, dim3 b, cudaStream_t s, const double *phi,
                     const double *psi, const double *C, const double *u);
    static void moments(const Inst<R> &I, dim3 g, dim3 b, cudaStream_t s);
    static void grad(const Inst<R> &I, dim3 g, dim3 b, cudaStream_t s, int guess = 1);
    static void force(const Inst<R> &I, dim3 g, dim3 b, cudaStream_t s);
    static void fd(const Inst<R> &I, dim3 g, dim3 b, cudaStream_t s, double *Sout,
                   double *Bout);
    static void collide(const Inst<R> &I, dim3 g, dim3 b, cudaStream_t s);
    static void stream(const Inst<R> &I, dim3 g, dim3 b, cudaStream_t s);
    static void diag(const Inst<R> &I, dim3 g, dim3 b, cudaStream_t s, int nblocks);
    // one red (colour 0) or black (colour 1) SOR half-sweep: variant 0 one
    // thread a cell (k_sor_rb3), variants 2 and 3 column marching through 8
    // or 4 planes (k_sor_cm3)
    static void sor(const Inst<R> &I, dim3 g, dim3 b, cudaStream_t s, int colour,
                    cudaGraphConditionalHandle h, int max_rounds, int eager_round,
                    int variant = 0);
    // the half-sweep kernel, for a kernel node of the SOR loop's body graph
    static void *sor_fn(int variant = 0);
    // grid of the half-sweep kernel of a variant (blocks of kSorBX x kSorBY)
    static dim3 sor_grid(int variant, int nx, int ny, int nz);
    static constexpr int kSorBX = 32, kSorBY = 8;
    // one full sweep with z-marching tiles (k_sor_zm3): kernel, grid,
    // threads and shared memory
    static void *zm_fn();
    static dim3 zm_grid(int nx, int ny, int nz);
    static int zm_threads();
    static size_t zm_smem();
};

}  // namespace lbs
