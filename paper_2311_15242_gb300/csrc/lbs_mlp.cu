// lbs_mlp.cu — the surrogate network: an ensemble of E fully connected
// networks n_in -> width (x depth hidden layers, SiLU) -> n_out (linear),
// trained by mean-squared error with Adam, evaluated with FP32 or bfloat16
// weights.  Every step of training and inference runs in the kernels below.
//
// Definitions (standard, stated here because the paper has no learned part):
//   SiLU(z) = z s(z), s(z) = 1 / (1 + exp(-z)), SiLU'(z) = s(z)(1 + z(1 - s(z)));
//   loss of a member = mean over the minibatch rows and outputs of (y - t)^2;
//   Adam (Kingma & Ba 2015): m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2,
//   theta <- theta - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
// Parameters of a member: for each layer l = 1..L, W_l (d_l x d_{l-1},
// row-major) then b_l (d_l); members follow each other.
//
// Layout: activations [E][B][d]; the minibatch of a member is drawn with
// replacement from the data set by SplitMix64 (Steele, Lea & Flood 2014)
// on (seed, iteration, member, row), so members see different minibatches.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/lbs.h"

namespace {

constexpr int kMaxWidth = 128;  // widest layer (threads of a block)
constexpr int kRows = 32;       // minibatch rows per block in the layer kernels
constexpr int kMaxLayers = 8;

struct Shape {
    int L;                        // weight layers
    int d[kMaxLayers + 1];        // d[0] = n_in, ..., d[L] = n_out
    long long woff[kMaxLayers + 1], boff[kMaxLayers + 1];  // offsets in a member's vector
    long long P;                  // parameters per member
};

__device__ __forceinline__ float tof(float x) { return x; }
__device__ __forceinline__ float tof(__nv_bfloat16 x) { return __bfloat162float(x); }

__device__ __forceinline__ float sigm(float z) { return 1.0f / (1.0f + expf(-z)); }
__device__ __forceinline__ float silu(float z) { return z * sigm(z); }
__device__ __forceinline__ float dsilu(float z) {
    const float s = sigm(z);
    return s * (1.0f + z * (1.0f - s));
}

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// minibatch of every member: rows drawn with replacement
__global__ void k_gather(const float *X, const float *Y, int n, int nin, int nout, int B, int E,
                         unsigned long long seed, long long iter, float *A0, float *T) {
    const int e = blockIdx.y;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x) {
        const unsigned long long key = ((unsigned long long)iter * E + e) * (unsigned long long)B + b;
        const int r = (int)(splitmix64(seed ^ splitmix64(key)) % (unsigned long long)n);
        for (int i = 0; i < nin; i++) A0[((long long)e * B + b) * nin + i] = X[(long long)r * nin + i];
        for (int o = 0; o < nout; o++) T[((long long)e * B + b) * nout + o] = Y[(long long)r * nout + o];
    }
}

// the same inputs for every member (inference)
__global__ void k_broadcast(const float *x, int n, int nin, int E, float *A0) {
    const int e = blockIdx.y;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n * nin; q += gridDim.x * blockDim.x)
        A0[(long long)e * n * nin + q] = x[q];
}

// Z_l = A_{l-1} W_l^T + b_l; A_l = SiLU(Z_l) (hidden) or Z_l (output).
// Block: kMaxWidth threads (output o = thread), kRows rows staged in shared
// memory; grid (row tiles, members).  WT: float or bf16 weights.
template <typename WT>
__global__ void __launch_bounds__(kMaxWidth)
    k_fwd(const WT *params, long long P, long long woff, long long boff, int din, int dout,
          int B, const float *Ain, float *Z, float *Aout, int hidden) {
    __shared__ float tile[kRows][kMaxWidth];
    const int e = blockIdx.y, r0 = blockIdx.x * kRows, o = threadIdx.x;
    const float *A = Ain + (long long)e * B * din;
    for (int q = threadIdx.x; q < kRows * din; q += blockDim.x) {
        const int r = q / din, i = q % din;
        tile[r][i] = (r0 + r < B) ? A[(long long)(r0 + r) * din + i] : 0.0f;
    }
    __syncthreads();
    if (o >= dout) return;
    const WT *W = params + (long long)e * P + woff + (long long)o * din;
    float acc[kRows];
    const float bias = tof(params[(long long)e * P + boff + o]);
#pragma unroll
    for (int r = 0; r < kRows; r++) acc[r] = bias;
    for (int i = 0; i < din; i++) {
        const float w = tof(W[i]);
#pragma unroll
        for (int r = 0; r < kRows; r++) acc[r] = fmaf(tile[r][i], w, acc[r]);
    }
    for (int r = 0; r < kRows; r++) {
        if (r0 + r >= B) break;
        const long long k = ((long long)e * B + r0 + r) * dout + o;
        if (Z) Z[k] = acc[r];
        Aout[k] = hidden ? silu(acc[r]) : acc[r];
    }
}

// loss of every member and dL/dy = 2 (y - t) / (B nout); one block a member,
// thread sums in a fixed order, then a fixed tree (deterministic)
__global__ void k_loss(const float *Yp, const float *T, int B, int nout, float *dY, double *loss) {
    const int e = blockIdx.x;
    const long long n = (long long)B * nout;
    const float sc = 2.0f / float(n);
    double s = 0.0;
    for (long long q = threadIdx.x; q < n; q += blockDim.x) {
        const long long k = (long long)e * n + q;
        const float d = Yp[k] - T[k];
        dY[k] = sc * d;
        s += double(d) * double(d);
    }
    __shared__ double sh[256];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) loss[e] = sh[0] / double(n);
}

// dZ_{l-1} = (dZ_l W_l) * SiLU'(Z_{l-1}); thread = input unit i, kRows rows
__global__ void __launch_bounds__(kMaxWidth)
    k_bwd_data(const float *params, long long P, long long woff, int din, int dout, int B,
               const float *dZ, const float *Zprev, float *dZprev) {
    __shared__ float tile[kRows][kMaxWidth];
    const int e = blockIdx.y, r0 = blockIdx.x * kRows, i = threadIdx.x;
    for (int q = threadIdx.x; q < kRows * dout; q += blockDim.x) {
        const int r = q / dout, o = q % dout;
        tile[r][o] = (r0 + r < B) ? dZ[((long long)e * B + r0 + r) * dout + o] : 0.0f;
    }
    __syncthreads();
    if (i >= din) return;
    const float *W = params + (long long)e * P + woff;
    float acc[kRows];
#pragma unroll
    for (int r = 0; r < kRows; r++) acc[r] = 0.0f;
    for (int o = 0; o < dout; o++) {
        const float w = W[(long long)o * din + i];
#pragma unroll
        for (int r = 0; r < kRows; r++) acc[r] = fmaf(tile[r][o], w, acc[r]);
    }
    for (int r = 0; r < kRows; r++) {
        if (r0 + r >= B) break;
        const long long k = ((long long)e * B + r0 + r) * din + i;
        dZprev[k] = acc[r] * dsilu(Zprev[k]);
    }
}

// dW_l[o][i] = sum_b dZ_l[b][o] A_{l-1}[b][i] (rows in order); db_l[o] =
// sum_b dZ_l[b][o].  Block: one output unit o, threads over i; grid (dout, E)
__global__ void __launch_bounds__(kMaxWidth)
    k_bwd_weight(long long P, long long woff, long long boff, int din, int dout, int B,
                 const float *dZ, const float *Aprev, float *grad) {
    const int e = blockIdx.y, o = blockIdx.x, i = threadIdx.x;
    const float *dz = dZ + (long long)e * B * dout;
    const float *a = Aprev + (long long)e * B * din;
    float *g = grad + (long long)e * P;
    if (i < din) {
        float s = 0.0f;
        for (int b = 0; b < B; b++) s = fmaf(dz[(long long)b * dout + o], a[(long long)b * din + i], s);
        g[woff + (long long)o * din + i] = s;
    }
    if (i == 0) {
        float s = 0.0f;
        for (int b = 0; b < B; b++) s += dz[(long long)b * dout + o];
        g[boff + o] = s;
    }
}

__global__ void k_adam(float *p, const float *g, float *m, float *v, long long n, float lr,
                       float b1, float b2, float eps, float c1, float c2) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const float gk = g[k];
        const float mk = b1 * m[k] + (1.0f - b1) * gk;
        const float vk = b2 * v[k] + (1.0f - b2) * gk * gk;
        m[k] = mk;
        v[k] = vk;
        p[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
    }
}

__global__ void k_to_bf16(const float *p, __nv_bfloat16 *q, long long n) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x)
        q[k] = __float2bfloat16_rn(p[k]);
}

// ensemble mean and standard deviation (population) over the E members
__global__ void k_stats(const float *Y, int E, long long n, float *mean, float *sd) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        double s = 0, s2 = 0;
        for (int e = 0; e < E; e++) s += Y[(long long)e * n + k];
        const double mu = s / E;
        for (int e = 0; e < E; e++) {
            const double d = Y[(long long)e * n + k] - mu;
            s2 += d * d;
        }
        mean[k] = float(mu);
        sd[k] = float(sqrt(s2 / E));
    }
}

// Glorot-uniform weights, zero biases, from SplitMix64 on (seed, index)
__global__ void k_init(float *p, long long n, const long long *woff, const long long *boff,
                       const int *d, int L, long long P, unsigned long long seed) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const long long q = k % P;
        float val = 0.0f;
        for (int l = 1; l <= L; l++) {
            if (q >= woff[l] && q < boff[l]) {
                const float a = sqrtf(6.0f / float(d[l - 1] + d[l]));
                const unsigned long long r = splitmix64(seed ^ splitmix64((unsigned long long)k));
                const float u = float((r >> 40) * (1.0 / 16777216.0));  // [0, 1), 24 bits
                val = (2.0f * u - 1.0f) * a;
            }
        }
        p[k] = val;
    }
}

}  // namespace

struct lbs_mlp {
    int E = 0, B = 0;
    Shape s;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    float *params = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    __nv_bfloat16 *pbf = nullptr;
    bool bf_valid = false;
    float *Z[kMaxLayers + 1] = {}, *A[kMaxLayers + 1] = {};
    float *dZa = nullptr, *dZb = nullptr, *T = nullptr, *stats = nullptr;
    double *loss = nullptr;
    float *X = nullptr, *Yd = nullptr;
    int ndata = 0;
    long long t = 0;  // Adam steps taken
    char err[512] = {0};

    ~lbs_mlp() {
        if (stream) cudaStreamSynchronize(stream);
        float *fl[] = {params, grad, m, v, dZa, dZb, T, stats, X, Yd};
        for (float *p : fl) cudaFree(p);
        for (int l = 0; l <= kMaxLayers; l++) {
            cudaFree(Z[l]);
            cudaFree(A[l]);
        }
        cudaFree(pbf);
        cudaFree(loss);
        if (own_stream && stream) cudaStreamDestroy(stream);
    }
};

namespace {

void merr(lbs_mlp *n, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(n->err, sizeof(n->err), fmt, ap);
    va_end(ap);
}

#define MCK(call)                                                                         \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            merr(net, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__,   \
                 __LINE__);                                                               \
            return LBS_ECUDA;                                                             \
        }                                                                                 \
    } while (0)

int forward(lbs_mlp *net, int B, bool bf16) {
    const Shape &s = net->s;
    for (int l = 1; l <= s.L; l++) {
        dim3 g((B + kRows - 1) / kRows, net->E);
        const int hidden = l < s.L;
        if (bf16)
            k_fwd<__nv_bfloat16><<<g, kMaxWidth, 0, net->stream>>>(
                net->pbf, s.P, s.woff[l], s.boff[l], s.d[l - 1], s.d[l], B, net->A[l - 1],
                net->Z[l], net->A[l], hidden);
        else
            k_fwd<float><<<g, kMaxWidth, 0, net->stream>>>(net->params, s.P, s.woff[l], s.boff[l],
                                                           s.d[l - 1], s.d[l], B, net->A[l - 1],
                                                           net->Z[l], net->A[l], hidden);
    }
    MCK(cudaGetLastError());
    return LBS_OK;
}

// loss and gradient of every member for the minibatch already in A[0], T
int backward(lbs_mlp *net, int B) {
    const Shape &s = net->s;
    k_loss<<<net->E, 256, 0, net->stream>>>(net->A[s.L], net->T, B, s.d[s.L], net->dZa, net->loss);
    float *dz = net->dZa, *dzp = net->dZb;
    for (int l = s.L; l >= 1; l--) {
        k_bwd_weight<<<dim3(s.d[l], net->E), kMaxWidth, 0, net->stream>>>(
            s.P, s.woff[l], s.boff[l], s.d[l - 1], s.d[l], B, dz, net->A[l - 1], net->grad);
        if (l > 1) {
            k_bwd_data<<<dim3((B + kRows - 1) / kRows, net->E), kMaxWidth, 0, net->stream>>>(
                net->params, s.P, s.woff[l], s.d[l - 1], s.d[l], B, dz, net->Z[l - 1], dzp);
            float *t = dz;
            dz = dzp;
            dzp = t;
        }
    }
    MCK(cudaGetLastError());
    return LBS_OK;
}

int adam(lbs_mlp *net, float lr, float b1, float b2, float eps) {
    net->t += 1;
    const float c1 = float(1.0 - std::pow(double(b1), double(net->t)));
    const float c2 = float(1.0 - std::pow(double(b2), double(net->t)));
    const long long n = (long long)net->E * net->s.P;
    k_adam<<<(int)std::min<long long>((n + 255) / 256, 4096), 256, 0, net->stream>>>(
        net->params, net->grad, net->m, net->v, n, lr, b1, b2, eps, c1, c2);
    net->bf_valid = false;
    MCK(cudaGetLastError());
    return LBS_OK;
}

int ensure_bf16(lbs_mlp *net) {
    if (net->bf_valid) return LBS_OK;
    const long long n = (long long)net->E * net->s.P;
    k_to_bf16<<<(int)std::min<long long>((n + 255) / 256, 4096), 256, 0, net->stream>>>(
        net->params, net->pbf, n);
    MCK(cudaGetLastError());
    net->bf_valid = true;
    return LBS_OK;
}

}  // namespace

extern "C" {

int lbs_mlp_create(int members, int n_in, int width, int depth, int n_out, int max_batch,
                   void *stream, lbs_mlp **out) {
    if (!out) return LBS_EINVAL;
    lbs_mlp *net = new (std::nothrow) lbs_mlp();
    *out = net;
    if (!net) return LBS_ENOMEM;
    if (members < 1 || n_in < 1 || n_out < 1 || width < 1 || depth < 1 || max_batch < 1 ||
        n_in > kMaxWidth || width > kMaxWidth || n_out > kMaxWidth || depth + 1 > kMaxLayers) {
        merr(net, "network %d -> %d x %d -> %d (E = %d, batch %d): widths 1..%d, depth 1..%d",
             n_in, width, depth, n_out, members, max_batch, kMaxWidth, kMaxLayers - 1);
        return LBS_EINVAL;
    }
    net->E = members;
    net->B = max_batch;
    Shape &s = net->s;
    s.L = depth + 1;
    s.d[0] = n_in;
    for (int l = 1; l <= depth; l++) s.d[l] = width;
    s.d[s.L] = n_out;
    long long off = 0;
    for (int l = 1; l <= s.L; l++) {
        s.woff[l] = off;
        off += (long long)s.d[l] * s.d[l - 1];
        s.boff[l] = off;
        off += s.d[l];
    }
    s.P = off;
    if (stream) {
        net->stream = (cudaStream_t)stream;
    } else {
        MCK(cudaStreamCreateWithFlags(&net->stream, cudaStreamNonBlocking));
        net->own_stream = true;
    }
    const long long EP = (long long)members * s.P;
    MCK(cudaMalloc(&net->params, EP * sizeof(float)));
    MCK(cudaMalloc(&net->grad, EP * sizeof(float)));
    MCK(cudaMalloc(&net->m, EP * sizeof(float)));
    MCK(cudaMalloc(&net->v, EP * sizeof(float)));
    MCK(cudaMalloc(&net->pbf, EP * sizeof(__nv_bfloat16)));
    MCK(cudaMemset(net->m, 0, EP * sizeof(float)));
    MCK(cudaMemset(net->v, 0, EP * sizeof(float)));
    MCK(cudaMemset(net->params, 0, EP * sizeof(float)));
    const long long EB = (long long)members * max_batch;
    for (int l = 0; l <= s.L; l++) {
        MCK(cudaMalloc(&net->A[l], EB * s.d[l] * sizeof(float)));
        if (l) MCK(cudaMalloc(&net->Z[l], EB * s.d[l] * sizeof(float)));
    }
    MCK(cudaMalloc(&net->dZa, EB * kMaxWidth * sizeof(float)));
    MCK(cudaMalloc(&net->dZb, EB * kMaxWidth * sizeof(float)));
    MCK(cudaMalloc(&net->T, EB * n_out * sizeof(float)));
    MCK(cudaMalloc(&net->stats, 2 * (long long)max_batch * n_out * sizeof(float)));
    MCK(cudaMalloc(&net->loss, members * sizeof(double)));
    return LBS_OK;
}

int lbs_mlp_param_count(const lbs_mlp *net) { return net ? (int)net->s.P : 0; }

int lbs_mlp_init(lbs_mlp *net, unsigned long long seed) {
    if (!net) return LBS_EINVAL;
    const Shape &s = net->s;
    long long *dw = nullptr;
    int *dd = nullptr;
    MCK(cudaMalloc(&dw, 2 * (kMaxLayers + 1) * sizeof(long long)));
    MCK(cudaMalloc(&dd, (kMaxLayers + 1) * sizeof(int)));
    MCK(cudaMemcpyAsync(dw, s.woff, (kMaxLayers + 1) * sizeof(long long), cudaMemcpyHostToDevice, net->stream));
    MCK(cudaMemcpyAsync(dw + kMaxLayers + 1, s.boff, (kMaxLayers + 1) * sizeof(long long),
                        cudaMemcpyHostToDevice, net->stream));
    MCK(cudaMemcpyAsync(dd, s.d, (kMaxLayers + 1) * sizeof(int), cudaMemcpyHostToDevice, net->stream));
    const long long n = (long long)net->E * s.P;
    k_init<<<(int)std::min<long long>((n + 255) / 256, 4096), 256, 0, net->stream>>>(
        net->params, n, dw, dw + kMaxLayers + 1, dd, s.L, s.P, seed);
    MCK(cudaGetLastError());
    MCK(cudaStreamSynchronize(net->stream));
    cudaFree(dw);
    cudaFree(dd);
    MCK(cudaMemsetAsync(net->m, 0, n * sizeof(float), net->stream));
    MCK(cudaMemsetAsync(net->v, 0, n * sizeof(float), net->stream));
    net->t = 0;
    net->bf_valid = false;
    return LBS_OK;
}

int lbs_mlp_set_params(lbs_mlp *net, const float *host) {
    if (!net || !host) return LBS_EINVAL;
    MCK(cudaMemcpyAsync(net->params, host, (long long)net->E * net->s.P * sizeof(float),
                        cudaMemcpyHostToDevice, net->stream));
    MCK(cudaStreamSynchronize(net->stream));
    net->bf_valid = false;
    return LBS_OK;
}

int lbs_mlp_get_params(lbs_mlp *net, float *host) {
    if (!net || !host) return LBS_EINVAL;
    MCK(cudaMemcpyAsync(host, net->params, (long long)net->E * net->s.P * sizeof(float),
                        cudaMemcpyDeviceToHost, net->stream));
    MCK(cudaStreamSynchronize(net->stream));
    return LBS_OK;
}

int lbs_mlp_forward(lbs_mlp *net, const float *x, int batch, int bf16, float *y) {
    if (!net || !x || !y || batch < 1 || batch > net->B) return LBS_EINVAL;
    const Shape &s = net->s;
    MCK(cudaMemcpyAsync(net->A[0], x, (long long)net->E * batch * s.d[0] * sizeof(float),
                        cudaMemcpyHostToDevice, net->stream));
    if (bf16) {
        int r = ensure_bf16(net);
        if (r) return r;
    }
    int r = forward(net, batch, bf16 != 0);
    if (r) return r;
    MCK(cudaMemcpyAsync(y, net->A[s.L], (long long)net->E * batch * s.d[s.L] * sizeof(float),
                        cudaMemcpyDeviceToHost, net->stream));
    MCK(cudaStreamSynchronize(net->stream));
    return LBS_OK;
}

int lbs_mlp_gradient(lbs_mlp *net, const float *x, const float *t, int batch, float *grad,
                     double *loss) {
    if (!net || !x || !t || batch < 1 || batch > net->B) return LBS_EINVAL;
    const Shape &s = net->s;
    MCK(cudaMemcpyAsync(net->A[0], x, (long long)net->E * batch * s.d[0] * sizeof(float),
                        cudaMemcpyHostToDevice, net->stream));
    MCK(cudaMemcpyAsync(net->T, t, (long long)net->E * batch * s.d[s.L] * sizeof(float),
                        cudaMemcpyHostToDevice, net->stream));
    int r = forward(net, batch, false);
    if (!r) r = backward(net, batch);
    if (r) return r;
    if (grad)
        MCK(cudaMemcpyAsync(grad, net->grad, (long long)net->E * s.P * sizeof(float),
                            cudaMemcpyDeviceToHost, net->stream));
    if (loss)
        MCK(cudaMemcpyAsync(loss, net->loss, net->E * sizeof(double), cudaMemcpyDeviceToHost,
                            net->stream));
    MCK(cudaStreamSynchronize(net->stream));
    return LBS_OK;
}

int lbs_mlp_set_grad(lbs_mlp *net, const float *host) {
    if (!net || !host) return LBS_EINVAL;
    MCK(cudaMemcpyAsync(net->grad, host, (long long)net->E * net->s.P * sizeof(float),
                        cudaMemcpyHostToDevice, net->stream));
    MCK(cudaStreamSynchronize(net->stream));
    return LBS_OK;
}

int lbs_mlp_adam_step(lbs_mlp *net, float lr, float beta1, float beta2, float eps) {
    if (!net || !(lr >= 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) ||
        !(eps > 0))
        return LBS_EINVAL;
    int r = adam(net, lr, beta1, beta2, eps);
    if (r) return r;
    MCK(cudaStreamSynchronize(net->stream));
    return LBS_OK;
}

int lbs_mlp_set_data(lbs_mlp *net, const float *X, const float *Y, int n) {
    if (!net || !X || !Y || n < 1) return LBS_EINVAL;
    cudaFree(net->X);
    cudaFree(net->Yd);
    net->X = net->Yd = nullptr;
    MCK(cudaMalloc(&net->X, (long long)n * net->s.d[0] * sizeof(float)));
    MCK(cudaMalloc(&net->Yd, (long long)n * net->s.d[net->s.L] * sizeof(float)));
    MCK(cudaMemcpyAsync(net->X, X, (long long)n * net->s.d[0] * sizeof(float),
                        cudaMemcpyHostToDevice, net->stream));
    MCK(cudaMemcpyAsync(net->Yd, Y, (long long)n * net->s.d[net->s.L] * sizeof(float),
                        cudaMemcpyHostToDevice, net->stream));
    MCK(cudaStreamSynchronize(net->stream));
    net->ndata = n;
    return LBS_OK;
}

int lbs_mlp_train(lbs_mlp *net, int iters, int batch, float lr, float beta1, float beta2,
                  float eps, unsigned long long seed, double *loss) {
    if (!net || iters < 0 || batch < 1 || batch > net->B || !net->X) return LBS_EINVAL;
    const Shape &s = net->s;
    for (int it = 0; it < iters; it++) {
        dim3 g((batch + 127) / 128, net->E);
        k_gather<<<g, 128, 0, net->stream>>>(net->X, net->Yd, net->ndata, s.d[0], s.d[s.L], batch,
                                             net->E, seed, net->t, net->A[0], net->T);
        int r = forward(net, batch, false);
        if (!r) r = backward(net, batch);
        if (!r) r = adam(net, lr, beta1, beta2, eps);
        if (r) return r;
    }
    if (loss)
        MCK(cudaMemcpyAsync(loss, net->loss, net->E * sizeof(double), cudaMemcpyDeviceToHost,
                            net->stream));
    MCK(cudaStreamSynchronize(net->stream));
    return LBS_OK;
}

int lbs_mlp_predict(lbs_mlp *net, const float *x, int n, int bf16, float *mean, float *sd) {
    if (!net || !x || !mean || !sd || n < 1) return LBS_EINVAL;
    const Shape &s = net->s;
    if (bf16) {
        int r = ensure_bf16(net);
        if (r) return r;
    }
    const int nout = s.d[s.L];
    for (int q0 = 0; q0 < n; q0 += net->B) {
        const int m = std::min(net->B, n - q0);
        float *xin = nullptr;
        MCK(cudaMalloc(&xin, (long long)m * s.d[0] * sizeof(float)));
        MCK(cudaMemcpyAsync(xin, x + (long long)q0 * s.d[0], (long long)m * s.d[0] * sizeof(float),
                            cudaMemcpyHostToDevice, net->stream));
        k_broadcast<<<dim3((m * s.d[0] + 255) / 256, net->E), 256, 0, net->stream>>>(
            xin, m, s.d[0], net->E, net->A[0]);
        int r = forward(net, m, bf16 != 0);
        if (r) {
            cudaFree(xin);
            return r;
        }
        const long long cnt = (long long)m * nout;
        k_stats<<<(int)((cnt + 255) / 256), 256, 0, net->stream>>>(net->A[s.L], net->E, cnt,
                                                                  net->stats, net->stats + cnt);
        MCK(cudaMemcpyAsync(mean + (long long)q0 * nout, net->stats, cnt * sizeof(float),
                            cudaMemcpyDeviceToHost, net->stream));
        MCK(cudaMemcpyAsync(sd + (long long)q0 * nout, net->stats + cnt, cnt * sizeof(float),
                            cudaMemcpyDeviceToHost, net->stream));
        MCK(cudaStreamSynchronize(net->stream));
        cudaFree(xin);
    }
    return LBS_OK;
}

void lbs_mlp_destroy(lbs_mlp *net) { delete net; }

const char *lbs_mlp_last_error(const lbs_mlp *net) {
    if (!net) return "null network";
    return net->err[0] ? net->err : "no error";
}

}  // extern "C"
