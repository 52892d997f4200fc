// Learned initial guess for the per-step GMRES solve (no counterpart in the paper).
//
// Per unknown m at step n: features x = (y_{n-1} .. y_{n-8})_m / s_n with s_n = RMS_m (y_{n-1})_m,
// network 8 -> 64 -> 64 -> 1 with tanh hidden layers, prediction y_{n,m} = y_{n-1,m} + s_n f(x) (the
// network learns the increment; a zero output is the previous-step guess).
// Parameters (FP32 master, 4801 floats): W1 (64 x 8), b1 (64), W2 (64 x 64), b2 (64), W3 (64), b3.
// Training: mini-batch squared error (1/2N) sum (f(x) - t)^2, gradient by these kernels (64-sample
// tiles in shared memory, per-block partial gradients added with atomics), Adam update.
// Inference (march and tdcfie_mlp_predict) uses FP16 copies of the weights with FP32 arithmetic.
#include <cuda_fp16.h>

#include <cmath>
#include <random>
#include <vector>

#include "gmres.h"
#include "plan.h"

namespace tdc {

constexpr int NIN = 8, NH = 64, NP = 4801;
constexpr int OW1 = 0, OB1 = 512, OW2 = 576, OB2 = 4672, OW3 = 4736, OB3 = 4800;
constexpr int TS = 64;   // samples per training tile

// dynamic shared memory of k_mlp_grad (floats): params, X tile, H1, H2, dZ2, dZ1, d
constexpr int GRAD_SMEM = (NP + 3) / 4 * 4 + TS * NIN + 4 * TS * NH + TS;

__global__ void k_mlp_grad(const float* __restrict__ prm, const float* __restrict__ X, const float* __restrict__ Y,
                           int64_t n, int64_t off, int64_t count, float inv_total, float* __restrict__ grad,
                           float* __restrict__ loss) {
    extern __shared__ float sm[];
    float* P = sm;
    float* Xs = P + (NP + 3) / 4 * 4;
    float* H1 = Xs + TS * NIN;
    float* H2 = H1 + TS * NH;
    float* D2 = H2 + TS * NH;
    float* D1 = D2 + TS * NH;
    float* dv = D1 + TS * NH;
    const int t = threadIdx.x;
    for (int i = t; i < NP; i += blockDim.x) P[i] = prm[i];
    const int64_t base = (int64_t)blockIdx.x * TS;
    for (int i = t; i < TS * NIN; i += blockDim.x) {
        const int64_t s = base + i / NIN;
        Xs[i] = s < count ? X[((off + s) % n) * NIN + i % NIN] : 0.f;
    }
    __syncthreads();
    for (int e = t; e < TS * NH; e += blockDim.x) {
        const int s = e / NH, i = e % NH;
        float z = P[OB1 + i];
        for (int k = 0; k < NIN; ++k) z += P[OW1 + i * NIN + k] * Xs[s * NIN + k];
        H1[e] = tanhf(z);
    }
    __syncthreads();
    for (int e = t; e < TS * NH; e += blockDim.x) {
        const int s = e / NH, i = e % NH;
        float z = P[OB2 + i];
        for (int j = 0; j < NH; ++j) z += P[OW2 + i * NH + j] * H1[s * NH + j];
        H2[e] = tanhf(z);
    }
    __syncthreads();
    if (t < TS) {
        const int64_t s = base + t;
        float o = P[OB3];
        for (int i = 0; i < NH; ++i) o += P[OW3 + i] * H2[t * NH + i];
        const float r = s < count ? o - Y[(off + s) % n] : 0.f;
        dv[t] = r * inv_total;
        atomicAdd(loss, 0.5f * r * r * inv_total);
    }
    __syncthreads();
    for (int e = t; e < TS * NH; e += blockDim.x) {
        const int s = e / NH, i = e % NH;
        D2[e] = dv[s] * P[OW3 + i] * (1.f - H2[e] * H2[e]);
    }
    __syncthreads();
    for (int e = t; e < TS * NH; e += blockDim.x) {
        const int s = e / NH, j = e % NH;
        float a = 0.f;
        for (int i = 0; i < NH; ++i) a += D2[s * NH + i] * P[OW2 + i * NH + j];
        D1[e] = a * (1.f - H1[e] * H1[e]);
    }
    __syncthreads();
    // block partial gradients
    for (int q = t; q < NP; q += blockDim.x) {
        float a = 0.f;
        if (q < OB1) {            // W1[i][k]
            const int i = q / NIN, k = q % NIN;
            for (int s = 0; s < TS; ++s) a += D1[s * NH + i] * Xs[s * NIN + k];
        } else if (q < OW2) {     // b1
            const int i = q - OB1;
            for (int s = 0; s < TS; ++s) a += D1[s * NH + i];
        } else if (q < OB2) {     // W2[i][j]
            const int i = (q - OW2) / NH, j = (q - OW2) % NH;
            for (int s = 0; s < TS; ++s) a += D2[s * NH + i] * H1[s * NH + j];
        } else if (q < OW3) {     // b2
            const int i = q - OB2;
            for (int s = 0; s < TS; ++s) a += D2[s * NH + i];
        } else if (q < OB3) {     // W3
            const int i = q - OW3;
            for (int s = 0; s < TS; ++s) a += dv[s] * H2[s * NH + i];
        } else {                  // b3
            for (int s = 0; s < TS; ++s) a += dv[s];
        }
        atomicAdd(grad + q, a);
    }
}

__global__ void k_mlp_adam(float* __restrict__ prm, const float* __restrict__ grad, float* __restrict__ m1,
                           float* __restrict__ m2, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= NP) return;
    const float g = grad[q];
    m1[q] = b1 * m1[q] + (1.f - b1) * g;
    m2[q] = b2 * m2[q] + (1.f - b2) * g * g;
    prm[q] -= lr * (m1[q] / c1) / (sqrtf(m2[q] / c2) + eps);
}

__global__ void k_to_half(const float* __restrict__ a, __half* __restrict__ b, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = __float2half_rn(a[i]);
}

// forward pass of one sample with FP16 weights staged in shared memory as FP32
__device__ __forceinline__ float mlp_forward(const float* P, const float* x) {
    float h1[NH];   // kept in registers: every loop that indexes it is fully unrolled
#pragma unroll
    for (int i = 0; i < NH; ++i) {
        float z = P[OB1 + i];
#pragma unroll
        for (int k = 0; k < NIN; ++k) z += P[OW1 + i * NIN + k] * x[k];
        h1[i] = tanhf(z);
    }
    float o = P[OB3];
    for (int i = 0; i < NH; ++i) {
        float z = P[OB2 + i];
#pragma unroll
        for (int j = 0; j < NH; ++j) z += P[OW2 + i * NH + j] * h1[j];
        o += P[OW3 + i] * tanhf(z);
    }
    return o;
}

__global__ void k_mlp_predict(const __half* __restrict__ wh, const float* __restrict__ X, int64_t n,
                              float* __restrict__ out) {
    __shared__ float P[NP];
    for (int i = threadIdx.x; i < NP; i += blockDim.x) P[i] = __half2float(wh[i]);
    __syncthreads();
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    float x[NIN];
    for (int k = 0; k < NIN; ++k) x[k] = X[s * NIN + k];
    out[s] = mlp_forward(P, x);
}

// RMS over ne entries of one vector, FP32 accumulation; block of 256 threads, result to all threads
// (1 for a zero vector).  Used both for the in-march guess and for training samples, so that the two
// scale their features identically.
template <typename T>
__device__ float block_rms(const T* __restrict__ y, int ne, float* red) {
    float a = 0.f;
    if (y)
        for (int i = threadIdx.x; i < ne; i += blockDim.x) a += (float)y[i] * (float)y[i];
    red[threadIdx.x] = a;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    const float s = sqrtf(red[0] / ne);
    __syncthreads();
    return s > 0.f ? s : 1.f;
}

// s_r = RMS over edges of y_{n-1} (one block of 256 threads per right-hand side)
template <typename T>
__global__ void k_mlp_rms(const T* __restrict__ ringbuf, int ring, int R, int ne, const Ctl* ctl,
                          float* __restrict__ scale) {
    __shared__ float red[256];
    const int r = blockIdx.x;
    const int64_t n = ctl->n;
    const T* y = n > 1 ? ringbuf + ((n - 1) % ring) * (int64_t)R * ne + (int64_t)r * ne : nullptr;
    const float s = block_rms(y, ne, red);
    if (threadIdx.x == 0) scale[r] = s;
}

// Training samples from a stored trajectory y (nt x R x ne, step-major): for t = 8 .. nt-1 the
// sample ((t - 8) R + r) ne + m has X = (y[t-1] .. y[t-8])_{r,m} / s and the increment target
// Y = (y[t] - base)_{r,m} / s with s = RMS_m y[t-1]_r, base y[t-1] or the cubic extrapolation
// 4 y[t-1] - 6 y[t-2] + 4 y[t-3] - y[t-4]; the difference is formed in the
// trajectory's own precision before the division, so small increments keep their digits.  One
// block of 256 threads per (t, r).
template <typename T>
__global__ void k_mlp_samples(const T* __restrict__ y, int R, int ne, int base, float* __restrict__ X,
                              float* __restrict__ Y) {
    __shared__ float red[256];
    const int64_t q = blockIdx.x;          // (t - 8) * R + r
    const int r = (int)(q % R);
    const int64_t t = q / R + 8;
    auto at = [&](int64_t step) { return y + (step * R + r) * (int64_t)ne; };
    const float s = block_rms(at(t - 1), ne, red);
    for (int m = threadIdx.x; m < ne; m += blockDim.x) {
        const int64_t o = q * ne + m;
        for (int k = 1; k <= NIN; ++k) X[o * NIN + k - 1] = (float)at(t - k)[m] / s;
        const T b = base ? (T)4 * at(t - 1)[m] - (T)6 * at(t - 2)[m] + (T)4 * at(t - 3)[m] - at(t - 4)[m] : at(t - 1)[m];
        Y[o] = (float)((at(t)[m] - b) / (T)s);
    }
}

// guess[r][m] = base + s_r f((y_{n-1..n-8})_{r,m} / s_r), base = y_{n-1} or (extrap) the cubic
// extrapolation 4 y_{n-1} - 6 y_{n-2} + 4 y_{n-3} - y_{n-4}; y_i = 0 for i <= 0.  The base is formed in
// the path precision T, so a network that outputs zero reproduces it exactly.
template <typename T>
__global__ void k_mlp_guess(const __half* __restrict__ wh, const T* __restrict__ ringbuf, int ring, int R, int ne,
                            const Ctl* ctl, const float* __restrict__ scale, int extrap, T* __restrict__ guess) {
    __shared__ float P[NP];
    for (int i = threadIdx.x; i < NP; i += blockDim.x) P[i] = __half2float(wh[i]);
    __syncthreads();
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= R * ne) return;
    const int r = idx / ne, m = idx % ne;
    const int64_t n = ctl->n;
    const float s = scale[r];
    float x[NIN];
    T yk[4] = {0, 0, 0, 0};
    for (int k = 1; k <= NIN; ++k) {
        T v = 0;
        if (n - k >= 1) {
            int64_t sl = (n - k) % ring;
            v = ringbuf[sl * (int64_t)R * ne + (int64_t)r * ne + m];
        }
        if (k <= 4) yk[k - 1] = v;
        x[k - 1] = (float)v / s;
    }
    const T base = extrap ? (T)4 * yk[0] - (T)6 * yk[1] + (T)4 * yk[2] - yk[3] : yk[0];
    guess[(int64_t)r * ne + m] = base + (T)(s * mlp_forward(P, x));   // base + predicted correction
}

// ---------------------------------------------------------------- march integration
struct MlpState {
    __half* wh = nullptr;
    float* scale = nullptr;
    bool loaded = false;
};

void destroy_mlp(MlpState* m) {
    if (!m) return;
    if (m->wh) cudaFree(m->wh);
    if (m->scale) cudaFree(m->scale);
    delete m;
}

template <typename T>
void launch_mlp_guess(StepPlan* p, cudaStream_t s) {
    MlpState* m = p->mlp;
    k_mlp_rms<T><<<p->R, 256, 0, s>>>((const T*)p->ringbuf, p->ring, p->R, p->ne, p->ctl, m->scale);
    k_mlp_guess<T><<<(p->R * p->ne + 127) / 128, 128, 0, s>>>(m->wh, (const T*)p->ringbuf, p->ring, p->R, p->ne,
                                                                p->ctl, m->scale, p->guess_extrap ? 1 : 0,
                                                                (T*)p->guessbuf);
    p->launches_per_step += 2;
}
template void launch_mlp_guess<double>(StepPlan*, cudaStream_t);
template void launch_mlp_guess<float>(StepPlan*, cudaStream_t);

cudaError_t build_mlp(StepPlan* p) {
    auto* m = new MlpState();
    p->mlp = m;
    cudaError_t e;
    if ((e = cudaMalloc(&m->wh, sizeof(__half) * NP)) != cudaSuccess) return e;
    if ((e = cudaMemset(m->wh, 0, sizeof(__half) * NP)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&m->scale, sizeof(float) * p->R)) != cudaSuccess) return e;
    return cudaSuccess;
}

cudaError_t mlp_load(StepPlan* p, const float* host_params, cudaStream_t s) {
    float* d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(float) * NP);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(d, host_params, sizeof(float) * NP, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        k_to_half<<<(NP + 255) / 256, 256, 0, s>>>(d, p->mlp->wh, NP);
        e = cudaStreamSynchronize(s);
    }
    cudaFree(d);
    p->mlp->loaded = (e == cudaSuccess);
    return e;
}

}  // namespace tdc

using namespace tdc;

static tdcfie_status launch_grad(const float* params, const float* X, const float* Y, int64_t n, int64_t off,
                                 int64_t count, float* grad, float* loss, cudaStream_t s) {
    // set on every call: the attribute is per device, and the call is cheap next to a training step
    const cudaError_t ea = cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                GRAD_SMEM * (int)sizeof(float));
    if (ea != cudaSuccess) return cuda_fail(nullptr, ea, "cudaFuncSetAttribute (MLP gradient)");
    const unsigned blocks = (unsigned)((count + TS - 1) / TS);
    k_mlp_grad<<<blocks, 256, GRAD_SMEM * sizeof(float), s>>>(params, X, Y, n, off, count, 1.f / (float)count, grad,
                                                              loss);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? TDCFIE_OK : cuda_fail(nullptr, e, "MLP gradient launch");
}

extern "C" tdcfie_status tdcfie_mlp_grad(const float* params, const float* X, const float* Y, int64_t n, float* grad,
                                         float* loss, void* stream) {
    if (!params || !X || !Y || !grad || !loss) return fail(nullptr, TDCFIE_E_ARG, "NULL device pointer");
    if (n < 1) return fail(nullptr, TDCFIE_E_ARG, "n must be >= 1");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(grad, 0, sizeof(float) * NP, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(loss, 0, sizeof(float), s);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaMemsetAsync");
    return launch_grad(params, X, Y, n, 0, n, grad, loss, s);
}

extern "C" tdcfie_status tdcfie_mlp_train(float* params, const float* X, const float* Y, int64_t n, int epochs,
                                          int64_t batch, float lr, uint64_t seed, float* loss_history, void* stream) {
    if (!params || !X || !Y) return fail(nullptr, TDCFIE_E_ARG, "NULL device pointer");
    if (n < 1 || epochs < 1 || batch < 1 || !(lr > 0.f)) return fail(nullptr, TDCFIE_E_ARG, "bad training sizes");
    cudaStream_t s = (cudaStream_t)stream;
    float* buf = nullptr;   // grad, m1, m2, loss
    cudaError_t e = cudaMallocAsync((void**)&buf, sizeof(float) * (3 * NP + 1), s);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaMallocAsync (MLP training state)");
    float *grad = buf, *m1 = buf + NP, *m2 = buf + 2 * NP, *loss = buf + 3 * NP;
    cudaMemsetAsync(buf, 0, sizeof(float) * (3 * NP + 1), s);
    std::mt19937_64 rng(seed);
    const int64_t nb = (n + batch - 1) / batch;
    int64_t step = 0;
    tdcfie_status st = TDCFIE_OK;
    for (int ep = 0; ep < epochs && st == TDCFIE_OK; ++ep) {
        const int64_t rot = (int64_t)(rng() % (uint64_t)n);   // per-epoch rotation of the batch origin
        cudaMemsetAsync(loss, 0, sizeof(float), s);
        for (int64_t b = 0; b < nb && st == TDCFIE_OK; ++b) {
            const int64_t off = (rot + b * batch) % n;
            const int64_t cnt = std::min<int64_t>(batch, n - b * batch);
            cudaMemsetAsync(grad, 0, sizeof(float) * NP, s);
            st = launch_grad(params, X, Y, n, off, cnt, grad, loss, s);
            ++step;
            const float c1 = 1.f - std::pow(0.9f, (float)step), c2 = 1.f - std::pow(0.999f, (float)step);
            k_mlp_adam<<<(NP + 255) / 256, 256, 0, s>>>(params, grad, m1, m2, lr, 0.9f, 0.999f, 1e-8f, c1, c2);
        }
        if (loss_history && st == TDCFIE_OK) {
            float l = 0.f;
            e = cudaMemcpyAsync(&l, loss, sizeof(float), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) st = cuda_fail(nullptr, e, "MLP loss readback");
            loss_history[ep] = l / (float)nb;
        }
    }
    cudaFreeAsync(buf, s);
    return st;
}

extern "C" tdcfie_status tdcfie_mlp_predict(const float* params, const float* X, int64_t n, float* out, void* stream) {
    if (!params || !X || !out) return fail(nullptr, TDCFIE_E_ARG, "NULL device pointer");
    if (n < 1) return fail(nullptr, TDCFIE_E_ARG, "n must be >= 1");
    cudaStream_t s = (cudaStream_t)stream;
    __half* wh = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&wh, sizeof(__half) * NP, s);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaMallocAsync (FP16 weights)");
    k_to_half<<<(NP + 255) / 256, 256, 0, s>>>(params, wh, NP);
    k_mlp_predict<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(wh, X, n, out);
    e = cudaGetLastError();
    cudaFreeAsync(wh, s);
    return e == cudaSuccess ? TDCFIE_OK : cuda_fail(nullptr, e, "MLP predict launch");
}

extern "C" tdcfie_status tdcfie_mlp_samples(int precision, int base, const void* y, int64_t nt, int64_t R,
                                            int64_t ne, float* X, float* Y, void* stream) {
    if (!y || !X || !Y) return fail(nullptr, TDCFIE_E_ARG, "NULL device pointer");
    if (precision != TDCFIE_FP64 && precision != TDCFIE_FP32) return fail(nullptr, TDCFIE_E_ARG, "y is float64 or float32");
    if (base != 0 && base != 1) return fail(nullptr, TDCFIE_E_ARG, "base is 0 (previous step) or 1 (extrapolation)");
    if (nt < 9 || R < 1 || ne < 1) return fail(nullptr, TDCFIE_E_ARG, "need nt >= 9, R >= 1, ne >= 1");
    if (ne > INT32_MAX || (nt - 8) * R > INT32_MAX) return fail(nullptr, TDCFIE_E_ARG, "sizes out of range");
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned blocks = (unsigned)((nt - 8) * R);
    if (precision == TDCFIE_FP64)
        k_mlp_samples<double><<<blocks, 256, 0, s>>>((const double*)y, (int)R, (int)ne, base, X, Y);
    else
        k_mlp_samples<float><<<blocks, 256, 0, s>>>((const float*)y, (int)R, (int)ne, base, X, Y);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? TDCFIE_OK : cuda_fail(nullptr, e, "MLP sample launch");
}

extern "C" tdcfie_status tdcfie_mlp_load(tdcfie_t h, const float* params) {
    if (!h || !params) return fail(h, TDCFIE_E_ARG, "NULL argument");
    if (!h->plan) return fail(h, TDCFIE_E_STATE, "call tdcfie_assemble first");
    if (h->plan->ring < 8) return fail(h, TDCFIE_E_UNSUPPORTED, "the learned guess needs K - 1 >= 8 stored steps");
    if (!h->plan->mlp) {
        const cudaError_t eb = build_mlp(h->plan);
        if (eb != cudaSuccess) return cuda_fail(h, eb, "learned-guess state");
    }
    const cudaError_t e = mlp_load(h->plan, params, h->stream);
    return e == cudaSuccess ? TDCFIE_OK : cuda_fail(h, e, "tdcfie_mlp_load");
}
