// lbs_3d.cu — instantiation and launchers of the D3Q19 kernels for the four
// population storage forms (FP64, FP32, FP16 and bfloat16 with FP32 arithmetic).
#include "lbs_k3d.cuh"
#include "lbs_launch3.h"

namespace lbs {

constexpr int kBS3 = Launch3<float, float>::kSorBX * Launch3<float, float>::kSorBY;

template <typename R, typename P>
void Launch3<R, P>::init(const Inst<R> &I, dim3 g, dim3 b, cudaStream_t s, const double *phi,
                         const double *psi, const double *C, const double *u) {
    k_init3<R, P><<<g, b, 0, s>>>(I, phi, psi, C, u);
}
template <typename R, typename P>
void Launch3<R, P>::moments(const Inst<R> &I, dim3 g, dim3 b, cudaStream_t s) {
    k_moments3<R, P><<<g, b, 0, s>>>(I);
}
template <typename R, typename P>
void Launch3<R, P>::grad(const Inst<R> &I, dim3 g, dim3 b, cudaStream_t s, int guess) {
    k_grad3<R><<<g, b, 0, s>>>(I, guess);
}
template <typename R, typename P>
void Launch3<R, P>::force(const Inst<R> &I, dim3 g, dim3 b, cudaStream_t s) {
    k_force3<R><<<g, b, 0, s>>>(I);
}
template <typename R, typename P>
void Launch3<R, P>::fd(const Inst<R> &I, dim3 g, dim3 b, cudaStream_t s, double *Sout,
                       double *Bout) {
    k_fd3<R><<<g, b, 0, s>>>(I, Sout, Bout);
}
template <typename R, typename P>
void Launch3<R, P>::collide(const Inst<R> &I, dim3 g, dim3 b, cudaStream_t s) {
    k_collide3<R, P><<<g, b, 0, s>>>(I);
}
template <typename R, typename P>
void Launch3<R, P>::stream(const Inst<R> &I, dim3 g, dim3 b, cudaStream_t s) {
    if (I.wall[0] == 2 || I.wall[1] == 2 || I.wall[2] == 2)
        k_stream3<R, P, true><<<g, b, 0, s>>>(I);
    else
        k_stream3<R, P, false><<<g, b, 0, s>>>(I);
}
template <typename R, typename P>
void Launch3<R, P>::diag(const Inst<R> &I, dim3 g, dim3 b, cudaStream_t s, int nblocks) {
    k_diag<R, P, 256, Q19><<<g, b, 0, s>>>(I, nblocks);
}
// column marching: planes a thread updates, 8 (variant 2) or 4 (variant 3,
// twice the blocks for grids that would not fill the GPU)
constexpr int cm_planes(int variant) { return variant == 3 ? 4 : 8; }

template <typename R, typename P>
void Launch3<R, P>::sor(const Inst<R> &I, dim3 g, dim3 b, cudaStream_t s, int colour,
                        cudaGraphConditionalHandle h, int max_rounds, int eager_round,
                        int variant) {
    if (variant == 2)
        k_sor_cm3<R, kBS3, 8><<<g, b, 0, s>>>(I, colour, h, max_rounds, eager_round);
    else if (variant == 3)
        k_sor_cm3<R, kBS3, 4><<<g, b, 0, s>>>(I, colour, h, max_rounds, eager_round);
    else
        k_sor_rb3<R, kBS3><<<g, b, 0, s>>>(I, colour, h, max_rounds, eager_round);
}
template <typename R, typename P>
void *Launch3<R, P>::sor_fn(int variant) {
    if (variant == 2) return (void *)k_sor_cm3<R, kBS3, 8>;
    if (variant == 3) return (void *)k_sor_cm3<R, kBS3, 4>;
    return (void *)k_sor_rb3<R, kBS3>;
}
template <typename R, typename P>
dim3 Launch3<R, P>::sor_grid(int variant, int nx, int ny, int nz) {
    const int hx = (nx + 1) / 2;  // cell pairs along x
    const dim3 g((hx + kSorBX - 1) / kSorBX, (ny + kSorBY - 1) / kSorBY, nz);
    if (variant == 2 || variant == 3) {
        const int zc = cm_planes(variant);
        return dim3(g.x, g.y, (nz + zc - 1) / zc);
    }
    return g;
}

constexpr int kZmTX = 32, kZmTY = 8, kZmZC = 16, kZmBS = 256;

template <typename R, typename P>
void *Launch3<R, P>::zm_fn() {
    return (void *)k_sor_zm3<R, kZmTX, kZmTY, kZmZC, kZmBS>;
}
template <typename R, typename P>
dim3 Launch3<R, P>::zm_grid(int nx, int ny, int nz) {
    return dim3((nx + kZmTX - 1) / kZmTX, (ny + kZmTY - 1) / kZmTY, (nz + kZmZC - 1) / kZmZC);
}
template <typename R, typename P>
int Launch3<R, P>::zm_threads() {
    return kZmBS;
}
template <typename R, typename P>
size_t Launch3<R, P>::zm_smem() {
    return SorZm<R, kZmTX, kZmTY, kZmZC, kZmBS>::smem_bytes();
}

template struct Launch3<double, double>;
template struct Launch3<float, float>;
template struct Launch3<float, __half>;
template struct Launch3<float, __nv_bfloat16>;

}  // namespace lbs
