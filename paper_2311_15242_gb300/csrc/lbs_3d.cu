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
    k_stream3<R, P><<<g, b, 0, s>>>(I);
}
template <typename R, typename P>
void Launch3<R, P>::diag(const Inst<R> &I, dim3 g, dim3 b, cudaStream_t s, int nblocks) {
    k_diag<R, P, 256, Q19><<<g, b, 0, s>>>(I, nblocks);
}
template <typename R, typename P>
void Launch3<R, P>::sor(const Inst<R> &I, dim3 g, dim3 b, cudaStream_t s, int colour,
                        cudaGraphConditionalHandle h, int max_rounds, int eager_round) {
    k_sor_rb3<R, kBS3><<<g, b, 0, s>>>(I, colour, h, max_rounds, eager_round);
}
template <typename R, typename P>
void *Launch3<R, P>::sor_fn() {
    return (void *)k_sor_rb3<R, kBS3>;
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
