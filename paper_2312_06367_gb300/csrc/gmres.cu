// Restarted GMRES on T_0 for the per-step solve T_0 y_n = b_n (Sec. IV-B), mixed precision:
//   restart: true residual r = b - T_0 x with T_0 in FP64 (the assembled block), convergence when
//            ||r|| <= tol ||b||;
//   cycle:   Arnoldi with the path-precision T_0 (FP32 or FP64 matvec), classical Gram-Schmidt
//            applied twice (CGS2) in FP64, Givens rotations, up to m iterations or until the
//            residual estimate drops below max(inner_tol beta, tol ||b|| / 2); then x += V_m y.
// Each right-hand side runs its own state machine (residual -> Arnoldi iterations -> update ->
// residual ...).  One pass of the loop body advances every open right-hand side by one Arnoldi
// iteration (plus, where due, its restart or update); the body sits in a CUDA-graph WHILE node whose
// condition the last kernel of the pass clears once every right-hand side has converged or given up
// (a pass cap bounds the loop).  No kernel waits on another.
#include <cmath>

#include "gmres.h"
#include "plan.h"

namespace tdc {

enum { F_DONE = 0, F_ST = 1, F_J = 2, F_ITERS = 3, NFLAGS = 4 };     // per right-hand side
enum { ST_ARN = 0, ST_RESID = 1, ST_UPD = 2 };                         // F_ST
enum { DONE_OPEN = 0, DONE_CONV = 1, DONE_GAVEUP = 2 };                // F_DONE
enum { S_BN2 = 0, S_RN2 = 1, S_WN2 = 2, S_BETA = 3, S_HN = 4, NSCAL = 6 };
// stats: [0] Arnoldi iterations this march, [1] steps, [2] max per step, [3] this step,
//        [4] solves not converged, [5] loop passes this march, [6] passes this step
enum { NSTATS = 8 };
constexpr int MV_WPB = 16;   // rows (warps) per block of the Arnoldi matvec

struct GmDev {
    int R, ne, m, maxit, pass_cap;
    double tol, inner_tol;
    double *x, *r, *V, *w, *hdot, *H, *cs, *sn, *g, *yv, *scal;
    int* flags;
    unsigned long long* stats;
};

__device__ __forceinline__ int fl(const GmDev& d, int r, int f) { return d.flags[r * NFLAGS + f]; }
__device__ __forceinline__ bool arnoldi(const GmDev& d, int r) {
    return fl(d, r, F_DONE) == DONE_OPEN && fl(d, r, F_ST) == ST_ARN;
}

// x = initial guess; ||b||^2; state reset; H cleared.  mode 0: zero, 1: y_{n-1} (ring slot
// (n-1) % ring), 2 and 4: the learned guess buffer, 3: cubic extrapolation of y_{n-1..n-4}
// (y_i = 0 for i <= 0)
template <typename T>
__global__ void k_gm_init(GmDev d, const T* __restrict__ b, int mode, const T* __restrict__ ringbuf, int ring,
                          const T* __restrict__ learned, const Ctl* ctl) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    const int64_t n = ctl->n;
    const T* guess = nullptr;
    if (mode == 1 && n > 1) guess = ringbuf + ((n - 1) % ring) * (int64_t)d.R * d.ne;
    if ((mode == 2 || mode == 4) && n > 1) guess = learned;
    if (i == 0) {
        d.flags[r * NFLAGS + F_DONE] = DONE_OPEN;
        d.flags[r * NFLAGS + F_ST] = ST_RESID;
        d.flags[r * NFLAGS + F_J] = 0;
        d.flags[r * NFLAGS + F_ITERS] = 0;
        d.scal[r * NSCAL + S_RN2] = 0.0;
        if (r == 0) { d.stats[3] = 0; d.stats[6] = 0; }
    }
    if (i < (d.m + 1) * d.m) d.H[(int64_t)r * (d.m + 1) * d.m + i] = 0.0;
    if (i < 2 * (d.m + 1)) d.hdot[(int64_t)r * 2 * (d.m + 1) + i] = 0.0;
    if (i >= d.ne) return;
    const double bi = (double)b[(int64_t)r * d.ne + i];
    double x0 = guess ? (double)guess[(int64_t)r * d.ne + i] : 0.0;
    if (mode == 3) {
        const double c[4] = {4.0, -6.0, 4.0, -1.0};
        x0 = 0.0;
        for (int k = 1; k <= 4 && k <= ring; ++k)
            if (n - k >= 1) x0 += c[k - 1] * (double)ringbuf[((n - k) % ring) * (int64_t)d.R * d.ne + (int64_t)r * d.ne + i];
    }
    d.x[(int64_t)r * d.ne + i] = x0;
    atomicAdd(d.scal + r * NSCAL + S_BN2, bi * bi);
}

__global__ void k_gm_zero_scal(GmDev d) {
    const int t = threadIdx.x;
    if (t < d.R * NSCAL) d.scal[t] = 0.0;
}

// r = b - T0 x (FP64 matrix), one warp per row, for a right-hand side at a restart (first pass of
// the step, or a cycle updated in the previous pass); accumulates ||r||^2
template <typename T>
__global__ void k_gm_resid(GmDev d, const double* __restrict__ T0, const T* __restrict__ b) {
    const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int r = blockIdx.y;
    if (row >= d.ne || fl(d, r, F_DONE) != DONE_OPEN || fl(d, r, F_ST) == ST_ARN) return;
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

// restart check: converged, out of iterations, or open a cycle with beta = ||r||
__global__ void k_gm_check(GmDev d) {
    const int r = threadIdx.x;
    if (r >= d.R || fl(d, r, F_DONE) != DONE_OPEN || fl(d, r, F_ST) == ST_ARN) return;
    double* sc = d.scal + r * NSCAL;
    const double beta = sqrt(sc[S_RN2]);
    const double bn = sqrt(sc[S_BN2]);
    sc[S_RN2] = 0.0;
    if (beta <= d.tol * bn || beta == 0.0) {
        d.flags[r * NFLAGS + F_DONE] = DONE_CONV;
        return;
    }
    if (fl(d, r, F_ITERS) >= d.maxit) {
        d.flags[r * NFLAGS + F_DONE] = DONE_GAVEUP;
        return;
    }
    sc[S_BETA] = beta;
    d.flags[r * NFLAGS + F_ST] = ST_ARN;
    d.flags[r * NFLAGS + F_J] = 0;
    double* g = d.g + (int64_t)r * (d.m + 1);
    g[0] = beta;
    for (int k = 1; k <= d.m; ++k) g[k] = 0.0;
}

// The block's contributions to hdot[k] = V_k . w (k <= j) for its nloc entries starting at i0, w of
// those entries in shared memory; one warp per k.
__device__ __forceinline__ void block_dots(const GmDev& d, int r, int j, int64_t i0, int nloc, const double* wsh,
                                           double* hdot) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = warp; k <= j; k += nw) {
        const double* v = d.V + ((int64_t)k * d.R + r) * d.ne + i0;
        double s = 0.0;
        for (int t = lane; t < nloc; t += 32) s += v[t] * wsh[t];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) atomicAdd(hdot + k, s);
    }
}

// Arnoldi iteration j, first part: w = T0p V_j (path precision matrix and accumulation, one warp per
// row) and the first Gram-Schmidt projections hdot0[k] = V_k . w.  A cycle opened in this pass
// (j = 0) takes V_0 = r / beta on the fly and stores it.
template <typename T, int WPB>
__global__ void __launch_bounds__(WPB * 32) k_gm_matvec(GmDev d, const T* __restrict__ T0p) {
    __shared__ double wsh[WPB];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r = blockIdx.y;
    if (!arnoldi(d, r)) return;
    const int j = fl(d, r, F_J);
    const int64_t row0 = (int64_t)blockIdx.x * WPB;
    const int64_t row = row0 + warp;
    const double* v = j == 0 ? d.r + (int64_t)r * d.ne : d.V + ((int64_t)j * d.R + r) * d.ne;
    const double sc = j == 0 ? 1.0 / d.scal[r * NSCAL + S_BETA] : 1.0;
    double wv = 0.0;
    if (row < d.ne) {
        const T* a = T0p + row * d.ne;
        T s = 0;
        for (int c = lane; c < d.ne; c += 32) s += a[c] * (T)(v[c] * sc);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        wv = (double)s;
        if (lane == 0) {
            d.w[(int64_t)r * d.ne + row] = wv;
            if (j == 0) d.V[(int64_t)r * d.ne + row] = v[row] * sc;
        }
    }
    if (lane == 0) wsh[warp] = wv;
    __syncthreads();   // also makes this block's V_0 stores visible to its warps
    const int nloc = (int)min((int64_t)WPB, d.ne - row0);
    block_dots(d, r, j, row0, nloc, wsh, d.hdot + (int64_t)r * 2 * (d.m + 1));
}

// w -= sum_k hdot[pass][k] V_k; pass 0 also accumulates the second projections hdot1 = V_k . w,
// pass 1 the norm ||w||^2
template <int PASS>
__global__ void __launch_bounds__(256) k_gm_orth(GmDev d) {
    __shared__ double hs[64];
    __shared__ double wsh[256];
    const int r = blockIdx.y;
    if (!arnoldi(d, r)) return;
    const int j = fl(d, r, F_J);
    const double* h = d.hdot + (int64_t)r * 2 * (d.m + 1) + PASS * (d.m + 1);
    for (int k = threadIdx.x; k <= j; k += blockDim.x) hs[k] = h[k];
    __syncthreads();
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x;
    const int64_t i = i0 + threadIdx.x;
    double v = 0.0;
    if (i < d.ne) {
        v = d.w[(int64_t)r * d.ne + i];
        for (int k = 0; k <= j; ++k) v -= hs[k] * d.V[((int64_t)k * d.R + r) * d.ne + i];
        d.w[(int64_t)r * d.ne + i] = v;
    }
    if (PASS == 0) {
        wsh[threadIdx.x] = v;
        __syncthreads();
        const int nloc = (int)min((int64_t)blockDim.x, d.ne - i0);
        block_dots(d, r, j, i0, nloc, wsh, d.hdot + (int64_t)r * 2 * (d.m + 1) + (d.m + 1));
    } else {
        double s = v * v;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(d.scal + r * NSCAL + S_WN2, s);
    }
}

// One thread per right-hand side: fold both projections into H[:, j] (clearing them), Givens update,
// residual estimate, cycle stop; at a stop, the back substitution H y = g.
__global__ void k_gm_givens(GmDev d) {
    const int r = threadIdx.x;
    if (r >= d.R || !arnoldi(d, r)) return;
    const int j = fl(d, r, F_J);
    double* H = d.H + (int64_t)r * (d.m + 1) * d.m;
    double* hd = d.hdot + (int64_t)r * 2 * (d.m + 1);
    double* cs = d.cs + (int64_t)r * (d.m + 1);
    double* sn = d.sn + (int64_t)r * (d.m + 1);
    double* g = d.g + (int64_t)r * (d.m + 1);
    double* sc = d.scal + r * NSCAL;
    for (int k = 0; k <= j; ++k) {
        H[(int64_t)k * d.m + j] = hd[k] + hd[d.m + 1 + k];
        hd[k] = 0.0;
        hd[d.m + 1 + k] = 0.0;
    }
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
    d.flags[r * NFLAGS + F_ITERS] += 1;
    atomicAdd(d.stats + 0, 1ULL);
    atomicAdd(d.stats + 3, 1ULL);
    // a cycle gains inner_tol, but never solves past half the outer target (the true FP64 residual
    // decides at the restart whether another cycle runs)
    const double goal = fmax(d.inner_tol * sc[S_BETA], 0.5 * d.tol * sqrt(sc[S_BN2]));
    const bool stop = fabs(g[j + 1]) <= goal || j + 1 == d.m || hn == 0.0 ||
                      fl(d, r, F_ITERS) >= d.maxit;
    sc[S_HN] = hn;    // kept for the next basis vector
    d.flags[r * NFLAGS + F_J] = j + 1;
    if (!stop) return;
    const int J = j + 1;
    double* y = d.yv + (int64_t)r * d.m;
    for (int i = J - 1; i >= 0; --i) {
        double t = g[i];
        for (int k = i + 1; k < J; ++k) t -= H[(int64_t)i * d.m + k] * y[k];
        y[i] = t / H[(int64_t)i * d.m + i];
    }
    d.flags[r * NFLAGS + F_ST] = ST_UPD;
}

// End of a pass, elementwise: V_{j+1} = w / h_{j+1,j} for a continuing cycle, x += V y and a
// cleared H for a finished one (whose ST_UPD state sends it to the restart of the next pass).  Thread 0 of block (0, 0) then
// sets the loop condition: another pass while some right-hand side is open, within the pass cap.
__global__ void __launch_bounds__(256) k_gm_finish(GmDev d, cudaGraphConditionalHandle cond) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (blockIdx.x == 0 && r == 0 && threadIdx.x == 0) {
        bool open = false;
        for (int q = 0; q < d.R; ++q) open |= fl(d, q, F_DONE) == DONE_OPEN;
        const unsigned long long passes = ++d.stats[6];
        d.stats[5] += 1;
        cudaGraphSetConditional(cond, (open && passes < (unsigned long long)d.pass_cap) ? 1u : 0u);
    }
    if (fl(d, r, F_DONE) != DONE_OPEN) return;
    const int st = fl(d, r, F_ST);
    const int J = fl(d, r, F_J);
    if (st == ST_ARN) {
        if (i < d.ne) d.V[((int64_t)J * d.R + r) * d.ne + i] = d.w[(int64_t)r * d.ne + i] / d.scal[r * NSCAL + S_HN];
    } else if (st == ST_UPD) {
        if (i < d.ne) {
            double v = d.x[(int64_t)r * d.ne + i];
            for (int k = 0; k < J; ++k) v += d.yv[(int64_t)r * d.m + k] * d.V[((int64_t)k * d.R + r) * d.ne + i];
            d.x[(int64_t)r * d.ne + i] = v;
        }
        if (i < (int64_t)(d.m + 1) * d.m) d.H[(int64_t)r * (d.m + 1) * d.m + i] = 0.0;
    }
}

// y_n (ring slot n % ring, path type) = x; statistics of the step; the first step with a solve
// left above the tolerance is recorded in the step state (returned as TDCFIE_E_NOCONV)
template <typename T>
__global__ void k_gm_store(GmDev d, T* __restrict__ ringbuf, int ring, Ctl* ctl) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (i == 0 && r == 0) {
        atomicAdd(d.stats + 1, 1ULL);
        atomicMax(d.stats + 2, d.stats[3]);
        for (int q = 0; q < d.R; ++q)
            if (fl(d, q, F_DONE) != DONE_CONV) {
                atomicAdd(d.stats + 4, 1ULL);
                if (atomicCAS(&ctl->noconv, 0, 1) == 0) ctl->noconv_step = ctl->n;
            }
    }
    if (i >= d.ne) return;
    T* dst = ringbuf + (ctl->n % ring) * (int64_t)d.R * d.ne;
    dst[(int64_t)r * d.ne + i] = (T)d.x[(int64_t)r * d.ne + i];
}

// ---------------------------------------------------------------- host side
struct GmresPlan {
    GmDev d{};
    cudaStream_t body_stream = nullptr;   // captures the loop body into the WHILE node's graph
    std::vector<void*> owned;
    ~GmresPlan() {
        for (void* p : owned) cudaFree(p);
        if (body_stream) cudaStreamDestroy(body_stream);
    }
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
    d.inner_tol = 1e-4;   // each cycle gains four digits; the restarts refine against the FP64 residual
    d.maxit = std::max(1, h->opts.gmres_maxit);
    // every pass performs one Arnoldi iteration of each open right-hand side, and each cycle ends
    // in one restart check that also starts the next cycle's first iteration
    d.pass_cap = d.maxit + d.maxit / m + 3;
    auto al = [&](double** q, size_t n) -> cudaError_t {
        cudaError_t e = cudaMalloc((void**)q, sizeof(double) * (n ? n : 1));
        if (e == cudaSuccess) { g->owned.push_back(*q); e = cudaMemset(*q, 0, sizeof(double) * (n ? n : 1)); }
        return e;
    };
    cudaError_t e;
    if ((e = al(&d.x, (size_t)R * ne)) || (e = al(&d.r, (size_t)R * ne)) || (e = al(&d.V, (size_t)(m + 1) * R * ne)) ||
        (e = al(&d.w, (size_t)R * ne)) || (e = al(&d.hdot, (size_t)R * 2 * (m + 1))) ||
        (e = al(&d.H, (size_t)R * (m + 1) * m)) || (e = al(&d.cs, (size_t)R * (m + 1))) ||
        (e = al(&d.sn, (size_t)R * (m + 1))) || (e = al(&d.g, (size_t)R * (m + 1))) || (e = al(&d.yv, (size_t)R * m)) ||
        (e = al(&d.scal, (size_t)R * NSCAL)))
        return e;
    if ((e = cudaMalloc(&d.flags, sizeof(int) * R * NFLAGS)) != cudaSuccess) return e;
    g->owned.push_back(d.flags);
    if ((e = cudaMemset(d.flags, 0, sizeof(int) * R * NFLAGS)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&d.stats, sizeof(unsigned long long) * NSTATS)) != cudaSuccess) return e;
    g->owned.push_back(d.stats);
    if ((e = cudaStreamCreateWithFlags(&g->body_stream, cudaStreamNonBlocking)) != cudaSuccess) return e;
    return cudaMemset(d.stats, 0, sizeof(unsigned long long) * NSTATS);
}

void gmres_set_tol(GmresPlan* g, double tol) { g->d.tol = tol; }

cudaError_t reset_gmres_stats(GmresPlan* g) { return cudaMemset(g->d.stats, 0, sizeof(unsigned long long) * NSTATS); }

cudaError_t gmres_stats(GmresPlan* g, long long* out6) {
    unsigned long long st[NSTATS];
    const cudaError_t e = cudaMemcpy(st, g->d.stats, sizeof(st), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return e;
    for (int i = 0; i < 6; ++i) out6[i] = (long long)st[i];
    return cudaSuccess;
}

// Kernels of one loop pass: resid, check, matvec, orth x 2, givens, finish
int gmres_body_launches() { return 7; }

// Enqueue the step's solve on s, which must be capturing a graph: init, the WHILE node (its body
// captured on the plan's own stream), then the store into the ring.
template <typename T>
cudaError_t launch_gmres(tdcfie_t h, StepPlan* p, const T* b, const T* learned, const T* T0p, T* ringbuf,
                         cudaStream_t s) {
    GmresPlan* g = p->gm;
    const GmDev& d = g->d;
    const int ne = d.ne, R = d.R, tb = 256, wpb = 8;
    const int ninit = std::max(ne, (d.m + 1) * d.m + 1);
    const dim3 gi((ninit + tb - 1) / tb, R), ge((ne + tb - 1) / tb, R), gw((ne + wpb - 1) / wpb, R),
        gm((ne + MV_WPB - 1) / MV_WPB, R);
    k_gm_zero_scal<<<1, 64, 0, s>>>(d);
    k_gm_init<T><<<gi, tb, 0, s>>>(d, b, h->opts.guess, ringbuf, p->ring, learned, p->ctl);

    cudaStreamCaptureStatus cs;
    cudaGraph_t graph = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* edata = nullptr;
    size_t ndeps = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &graph, &deps, &edata, &ndeps);
    if (e != cudaSuccess) return e;
    if (cs != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureUnmatched;
    cudaGraphConditionalHandle cond;
    if ((e = cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault)) != cudaSuccess) return e;
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = cond;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    if ((e = cudaGraphAddNode(&node, graph, deps, edata, ndeps, &np)) != cudaSuccess) return e;
    cudaGraph_t body = np.conditional.phGraph_out[0];
    if ((e = cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies)) !=
        cudaSuccess)
        return e;

    cudaStream_t b2 = g->body_stream;
    if ((e = cudaStreamBeginCaptureToGraph(b2, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed)) !=
        cudaSuccess)
        return e;
    k_gm_resid<T><<<gw, 32 * wpb, 0, b2>>>(d, h->T, b);
    k_gm_check<<<1, 32 * ((R + 31) / 32), 0, b2>>>(d);
    k_gm_matvec<T, MV_WPB><<<gm, 32 * MV_WPB, 0, b2>>>(d, T0p);
    k_gm_orth<0><<<ge, tb, 0, b2>>>(d);
    k_gm_orth<1><<<ge, tb, 0, b2>>>(d);
    k_gm_givens<<<1, 32 * ((R + 31) / 32), 0, b2>>>(d);
    k_gm_finish<<<gi, tb, 0, b2>>>(d, cond);
    cudaGraph_t captured = nullptr;
    const cudaError_t le = cudaGetLastError();
    if ((e = cudaStreamEndCapture(b2, &captured)) != cudaSuccess) return e;
    if (le != cudaSuccess) return le;

    k_gm_store<T><<<ge, tb, 0, s>>>(d, ringbuf, p->ring, p->ctl);
    p->launches_per_step += 3;   // zero_scal, init, store; the loop passes are counted on the device
    return cudaGetLastError();
}

template cudaError_t launch_gmres<double>(tdcfie_t, StepPlan*, const double*, const double*, const double*, double*,
                                          cudaStream_t);
template cudaError_t launch_gmres<float>(tdcfie_t, StepPlan*, const float*, const float*, const float*, float*,
                                         cudaStream_t);

}  // namespace tdc
