// Restarted GMRES on T_0 for the per-step solve T_0 y_n = b_n (Sec. IV-B), mixed precision:
//   outer cycle: true residual r = b - T_0 x with T_0 in FP64 (the assembled block), convergence when
//                ||r|| <= tol ||b||;
//   inner cycle: Arnoldi with the path-precision T_0 (FP32 or FP64 matvec), classical Gram-Schmidt
//                applied twice (CGS2) in FP64, Givens rotations, up to m iterations or until the
//                residual estimate drops below inner_tol * beta; x += V_m y.
// Every kernel reads per-right-hand-side flags and returns at once when its right-hand side has
// converged, so the fixed schedule (outer cycles x inner iterations) captured in the step graph
// costs only launch latency after convergence.  No kernel waits on another.
#include <cmath>

#include "gmres.h"
#include "plan.h"

namespace tdc {

enum { F_DONE = 0, F_INNER = 1, F_J = 2, F_ITERS = 3, NFLAGS = 4 };
enum { S_BN2 = 0, S_RN2 = 1, S_WN2 = 2, S_BETA = 3, S_HN = 4, NSCAL = 6 };

struct GmDev {
    int R, ne, m;
    double tol, inner_tol;
    double *x, *r, *V, *w, *hdot, *H, *cs, *sn, *g, *yv, *scal;
    int* flags;
    unsigned long long* stats;   // [0] inner iterations this march, [1] steps, [2] max per step, [3] this step
};

__device__ __forceinline__ bool active(const GmDev& d, int r) { return d.flags[r * NFLAGS + F_DONE] == 0; }
__device__ __forceinline__ bool inner_active(const GmDev& d, int r) {
    return d.flags[r * NFLAGS + F_DONE] == 0 && d.flags[r * NFLAGS + F_INNER] == 0;
}

// x = initial guess; ||b||^2; flags reset.  mode 0: zero, 1: y_{n-1} (ring slot (n-1) % ring),
// 2: the learned guess buffer
template <typename T>
__global__ void k_gm_init(GmDev d, const T* __restrict__ b, int mode, const T* __restrict__ ringbuf, int ring,
                          const T* __restrict__ learned, const Ctl* ctl) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    const int64_t n = ctl->n;
    const T* guess = nullptr;
    if (mode == 1 && n > 1) guess = ringbuf + ((n - 1) % ring) * (int64_t)d.R * d.ne;
    if (mode == 2 && n > 1) guess = learned;
    if (i == 0) {
        d.flags[r * NFLAGS + F_DONE] = 0;
        d.flags[r * NFLAGS + F_INNER] = 1;   // no inner cycle until an outer check opens one
        d.scal[r * NSCAL + S_RN2] = 0.0;
        if (r == 0) d.stats[3] = 0;
    }
    if (i >= d.ne) return;
    const double bi = (double)b[(int64_t)r * d.ne + i];
    d.x[(int64_t)r * d.ne + i] = guess ? (double)guess[(int64_t)r * d.ne + i] : 0.0;
    atomicAdd(d.scal + r * NSCAL + S_BN2, bi * bi);
}

__global__ void k_gm_zero_scal(GmDev d) {
    const int t = threadIdx.x;
    if (t < d.R * NSCAL) d.scal[t] = 0.0;
}

// r = b - T0 x (FP64 matrix), one warp per row; accumulates ||r||^2
template <typename T>
__global__ void k_gm_resid(GmDev d, const double* __restrict__ T0, const T* __restrict__ b) {
    const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int r = blockIdx.y;
    if (row >= d.ne || !active(d, r)) return;
    const double* a = T0 + (int64_t)row * d.ne;
    const double* xr = d.x + (int64_t)r * d.ne;
    double s = 0.0;
    for (int j = lane; j < d.ne; j += 32) s += a[j] * xr[j];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
        const double v = (double)b[(int64_t)r * d.ne + row] - s;
        d.r[(int64_t)r * d.ne + row] = v;
        atomicAdd(d.scal + r * NSCAL + S_RN2, v * v);
    }
}

// outer check: converged? else open an inner cycle with beta = ||r||
__global__ void k_gm_check(GmDev d) {
    const int r = threadIdx.x;
    if (r >= d.R || !active(d, r)) return;
    double* sc = d.scal + r * NSCAL;
    const double beta = sqrt(sc[S_RN2]);
    const double bn = sqrt(sc[S_BN2]);
    sc[S_RN2] = 0.0;
    if (beta <= d.tol * bn || beta == 0.0) {
        d.flags[r * NFLAGS + F_DONE] = 1;
        return;
    }
    sc[S_BETA] = beta;
    d.flags[r * NFLAGS + F_INNER] = 0;
    d.flags[r * NFLAGS + F_J] = 0;
    double* g = d.g + (int64_t)r * (d.m + 1);
    g[0] = beta;
    for (int k = 1; k <= d.m; ++k) g[k] = 0.0;
}

// V_0 = r / beta
__global__ void k_gm_v0(GmDev d) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (i >= d.ne || !inner_active(d, r)) return;
    d.V[(int64_t)r * d.ne + i] = d.r[(int64_t)r * d.ne + i] / d.scal[r * NSCAL + S_BETA];
}

// w = T0p V_j (path precision matrix, FP32 accumulation for float), one warp per row
template <typename T>
__global__ void k_gm_matvec(GmDev d, const T* __restrict__ T0p, int j) {
    const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int r = blockIdx.y;
    if (row >= d.ne || !inner_active(d, r) || d.flags[r * NFLAGS + F_J] != j) return;
    const T* a = T0p + (int64_t)row * d.ne;
    const double* v = d.V + ((int64_t)j * d.R + r) * d.ne;
    T s = 0;
    for (int c = lane; c < d.ne; c += 32) s += a[c] * (T)v[c];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) d.w[(int64_t)r * d.ne + row] = (double)s;
}

// hdot[i] = V_i . w for i <= j (block partial sums + atomics); hdot zeroed by the caller's prior kernel
__global__ void k_gm_dots(GmDev d, int j) {
    const int r = blockIdx.y;
    if (!inner_active(d, r) || d.flags[r * NFLAGS + F_J] != j) return;
    __shared__ double red[256];
    for (int i = 0; i <= j; ++i) {
        double s = 0.0;
        const double* v = d.V + ((int64_t)i * d.R + r) * d.ne;
        const double* w = d.w + (int64_t)r * d.ne;
        for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < d.ne; e += gridDim.x * blockDim.x) s += v[e] * w[e];
        red[threadIdx.x] = s;
        __syncthreads();
        for (int k = blockDim.x / 2; k > 0; k >>= 1) {
            if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
            __syncthreads();
        }
        if (threadIdx.x == 0) atomicAdd(d.hdot + (int64_t)r * (d.m + 1) + i, red[0]);
        __syncthreads();
    }
}

// w -= sum_i hdot[i] V_i ; H[:, j] += hdot ; hdot = 0 (second pass of CGS2 reuses it); ||w||^2 on pass 2
__global__ void k_gm_orth(GmDev d, int j, int pass) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (!inner_active(d, r) || d.flags[r * NFLAGS + F_J] != j) return;
    const double* h = d.hdot + (int64_t)r * (d.m + 1);
    if (i < d.ne) {
        double v = d.w[(int64_t)r * d.ne + i];
        for (int k = 0; k <= j; ++k) v -= h[k] * d.V[((int64_t)k * d.R + r) * d.ne + i];
        d.w[(int64_t)r * d.ne + i] = v;
        if (pass == 1) atomicAdd(d.scal + r * NSCAL + S_WN2, v * v);
    }
}

// fold hdot into H[:, j] and clear it (one block per right-hand side)
__global__ void k_gm_fold(GmDev d, int j) {
    const int r = blockIdx.x;
    if (!inner_active(d, r) || d.flags[r * NFLAGS + F_J] != j) return;
    double* h = d.hdot + (int64_t)r * (d.m + 1);
    double* H = d.H + (int64_t)r * (d.m + 1) * d.m;
    for (int k = threadIdx.x; k <= j; k += blockDim.x) {
        H[(int64_t)k * d.m + j] += h[k];
        h[k] = 0.0;
    }
}

// Givens update of column j, residual estimate, inner stop; one thread per right-hand side
__global__ void k_gm_givens(GmDev d, int j) {
    const int r = threadIdx.x;
    if (r >= d.R || !inner_active(d, r) || d.flags[r * NFLAGS + F_J] != j) return;
    double* H = d.H + (int64_t)r * (d.m + 1) * d.m;
    double* cs = d.cs + (int64_t)r * (d.m + 1);
    double* sn = d.sn + (int64_t)r * (d.m + 1);
    double* g = d.g + (int64_t)r * (d.m + 1);
    double* sc = d.scal + r * NSCAL;
    const double hn = sqrt(sc[S_WN2]);
    sc[S_WN2] = 0.0;
    H[(int64_t)(j + 1) * d.m + j] = hn;
    for (int k = 0; k < j; ++k) {
        const double a = H[(int64_t)k * d.m + j], b = H[(int64_t)(k + 1) * d.m + j];
        H[(int64_t)k * d.m + j] = cs[k] * a + sn[k] * b;
        H[(int64_t)(k + 1) * d.m + j] = -sn[k] * a + cs[k] * b;
    }
    const double a = H[(int64_t)j * d.m + j], b = H[(int64_t)(j + 1) * d.m + j];
    const double rr = sqrt(a * a + b * b);
    const double c = rr > 0.0 ? a / rr : 1.0, s = rr > 0.0 ? b / rr : 0.0;
    cs[j] = c;
    sn[j] = s;
    H[(int64_t)j * d.m + j] = rr;
    H[(int64_t)(j + 1) * d.m + j] = 0.0;
    g[j + 1] = -s * g[j];
    g[j] = c * g[j];
    sc[S_RN2] = 0.0;
    d.flags[r * NFLAGS + F_ITERS] += 1;
    atomicAdd(d.stats + 0, 1ULL);
    atomicAdd(d.stats + 3, 1ULL);
    // a cycle gains inner_tol, but never solves past half the outer target (the true FP64 residual
    // decides in k_gm_check whether another cycle runs)
    const double goal = fmax(d.inner_tol * sc[S_BETA], 0.5 * d.tol * sqrt(sc[S_BN2]));
    const bool stop = fabs(g[j + 1]) <= goal || j + 1 == d.m || hn == 0.0;
    sc[S_HN] = hn;    // kept for the next basis vector
    d.flags[r * NFLAGS + F_J] = j + 1;
    if (stop) d.flags[r * NFLAGS + F_INNER] = 2;   // 2: inner cycle finished, update pending
}

// V_{j+1} = w / h_{j+1,j}
__global__ void k_gm_next(GmDev d, int j) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (i >= d.ne || !inner_active(d, r) || d.flags[r * NFLAGS + F_J] != j + 1) return;
    d.V[((int64_t)(j + 1) * d.R + r) * d.ne + i] = d.w[(int64_t)r * d.ne + i] / d.scal[r * NSCAL + S_HN];
}

// back substitution H(0:J,0:J) y = g(0:J), one thread per right-hand side
__global__ void k_gm_small(GmDev d) {
    const int r = threadIdx.x;
    if (r >= d.R || d.flags[r * NFLAGS + F_DONE] != 0 || d.flags[r * NFLAGS + F_INNER] != 2) return;
    const int J = d.flags[r * NFLAGS + F_J];
    const double* H = d.H + (int64_t)r * (d.m + 1) * d.m;
    const double* g = d.g + (int64_t)r * (d.m + 1);
    double* y = d.yv + (int64_t)r * d.m;
    for (int i = J - 1; i >= 0; --i) {
        double s = g[i];
        for (int k = i + 1; k < J; ++k) s -= H[(int64_t)i * d.m + k] * y[k];
        y[i] = s / H[(int64_t)i * d.m + i];
    }
}

// x += V y; then H, hdot cleared for the next cycle; inner closed
__global__ void k_gm_update(GmDev d) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (d.flags[r * NFLAGS + F_DONE] != 0 || d.flags[r * NFLAGS + F_INNER] != 2) return;
    const int J = d.flags[r * NFLAGS + F_J];
    if (i < d.ne) {
        double v = d.x[(int64_t)r * d.ne + i];
        for (int k = 0; k < J; ++k) v += d.yv[(int64_t)r * d.m + k] * d.V[((int64_t)k * d.R + r) * d.ne + i];
        d.x[(int64_t)r * d.ne + i] = v;
    }
}

__global__ void k_gm_close(GmDev d) {
    const int r = blockIdx.x;
    if (d.flags[r * NFLAGS + F_DONE] != 0 || d.flags[r * NFLAGS + F_INNER] != 2) return;
    double* H = d.H + (int64_t)r * (d.m + 1) * d.m;
    for (int k = threadIdx.x; k < (d.m + 1) * d.m; k += blockDim.x) H[k] = 0.0;
    __syncthreads();
    if (threadIdx.x == 0) d.flags[r * NFLAGS + F_INNER] = 1;
}

// y_n (ring slot n % ring, path type) = x; statistics of the step
template <typename T>
__global__ void k_gm_store(GmDev d, T* __restrict__ ringbuf, int ring, const Ctl* ctl) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (i == 0 && r == 0) {
        atomicAdd(d.stats + 1, 1ULL);
        atomicMax(d.stats + 2, d.stats[3]);
        // a right-hand side still open after the last outer cycle did not converge
        for (int q = 0; q < d.R; ++q)
            if (d.flags[q * NFLAGS + F_DONE] == 0) atomicAdd(d.stats + 4, 1ULL);
    }
    if (i >= d.ne) return;
    T* dst = ringbuf + (ctl->n % ring) * (int64_t)d.R * d.ne;
    dst[(int64_t)r * d.ne + i] = (T)d.x[(int64_t)r * d.ne + i];
}

// ---------------------------------------------------------------- host side
struct GmresPlan {
    GmDev d{};
    int outer = 3;
    std::vector<void*> owned;
    ~GmresPlan() { for (void* p : owned) cudaFree(p); }
};

void destroy_gmres(GmresPlan* g) { delete g; }

cudaError_t build_gmres(tdcfie_t h, StepPlan* p) {
    auto* g = new GmresPlan();
    p->gm = g;
    const int R = p->R, ne = p->ne;
    const int m = std::max(2, std::min(60, h->opts.gmres_restart));
    GmDev& d = g->d;
    d.R = R; d.ne = ne; d.m = m;
    d.tol = h->opts.gmres_tol;
    d.inner_tol = 1e-4;   // each inner cycle gains four digits; the outer cycles refine in FP64
    g->outer = std::max(1, std::min(8, h->opts.gmres_maxit / m + 1));
    auto al = [&](double** q, size_t n) -> cudaError_t {
        cudaError_t e = cudaMalloc((void**)q, sizeof(double) * (n ? n : 1));
        if (e == cudaSuccess) { g->owned.push_back(*q); e = cudaMemset(*q, 0, sizeof(double) * (n ? n : 1)); }
        return e;
    };
    cudaError_t e;
    if ((e = al(&d.x, (size_t)R * ne)) || (e = al(&d.r, (size_t)R * ne)) || (e = al(&d.V, (size_t)(m + 1) * R * ne)) ||
        (e = al(&d.w, (size_t)R * ne)) || (e = al(&d.hdot, (size_t)R * (m + 1))) ||
        (e = al(&d.H, (size_t)R * (m + 1) * m)) || (e = al(&d.cs, (size_t)R * (m + 1))) ||
        (e = al(&d.sn, (size_t)R * (m + 1))) || (e = al(&d.g, (size_t)R * (m + 1))) || (e = al(&d.yv, (size_t)R * m)) ||
        (e = al(&d.scal, (size_t)R * NSCAL)))
        return e;
    if ((e = cudaMalloc(&d.flags, sizeof(int) * R * NFLAGS)) != cudaSuccess) return e;
    g->owned.push_back(d.flags);
    if ((e = cudaMalloc(&d.stats, sizeof(unsigned long long) * 8)) != cudaSuccess) return e;
    g->owned.push_back(d.stats);
    return cudaMemset(d.stats, 0, sizeof(long long) * 8);
}

cudaError_t reset_gmres_stats(GmresPlan* g) { return cudaMemset(g->d.stats, 0, sizeof(long long) * 8); }

cudaError_t gmres_stats(GmresPlan* g, long long* out5) {
    return cudaMemcpy(out5, g->d.stats, sizeof(long long) * 5, cudaMemcpyDeviceToHost);
}

template <typename T>
void launch_gmres(tdcfie_t h, StepPlan* p, const T* b, const T* learned, const T* T0p, T* ringbuf, cudaStream_t s) {
    GmresPlan* g = p->gm;
    const GmDev& d = g->d;
    const int ne = d.ne, R = d.R, tb = 256, wpb = 8;
    const dim3 ge((ne + tb - 1) / tb, R), gw((ne + wpb - 1) / wpb, R), gd(std::min(64, (ne + tb - 1) / tb), R);
    k_gm_zero_scal<<<1, 64, 0, s>>>(d);
    k_gm_init<T><<<ge, tb, 0, s>>>(d, b, h->opts.guess, ringbuf, p->ring, learned, p->ctl);
    for (int o = 0; o < g->outer; ++o) {
        k_gm_resid<T><<<gw, 32 * wpb, 0, s>>>(d, h->T, b);
        k_gm_check<<<1, 32, 0, s>>>(d);
        k_gm_v0<<<ge, tb, 0, s>>>(d);
        for (int j = 0; j < d.m; ++j) {
            k_gm_matvec<T><<<gw, 32 * wpb, 0, s>>>(d, T0p, j);
            for (int pass = 0; pass < 2; ++pass) {
                k_gm_dots<<<gd, tb, 0, s>>>(d, j);
                k_gm_orth<<<ge, tb, 0, s>>>(d, j, pass);
                k_gm_fold<<<R, 32, 0, s>>>(d, j);
            }
            k_gm_givens<<<1, 32, 0, s>>>(d, j);
            k_gm_next<<<ge, tb, 0, s>>>(d, j);
        }
        k_gm_small<<<1, 32, 0, s>>>(d);
        k_gm_update<<<ge, tb, 0, s>>>(d);
        k_gm_close<<<R, 128, 0, s>>>(d);
    }
    k_gm_store<T><<<ge, tb, 0, s>>>(d, ringbuf, p->ring, p->ctl);
    p->launches_per_step += 3 + g->outer * (5 + d.m * 9) + 1;
}

template void launch_gmres<double>(tdcfie_t, StepPlan*, const double*, const double*, const double*, double*,
                                   cudaStream_t);
template void launch_gmres<float>(tdcfie_t, StepPlan*, const float*, const float*, const float*, float*,
                                  cudaStream_t);

}  // namespace tdc
