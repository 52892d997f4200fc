// Hot path of the marching-on-in-time solver (Sec. IV-B), one CUDA graph per step.
//
// Per step n (t_n = n dt), with y_i = 0 for i <= 0:
//   rhs:      e_m(t_n) = int f_m . e_in(t_n),  h_m(t_n) = int g_m . h_in(t_n)         (Sec. II-C)
//   history:  b_n = -A e_n + alpha L2 h_n - sum_{k=1}^{K-1} T_k y_{n-k}                 (Sec. IV-B)
//             A = L1 (dtt P^LH + P^S) folds the rescaling of e (Sec. III-A) into L1
//   solve:    y_n = T_0^-1 b_n
//   project:  z = Sigma^T w_n, w_n = (1/dtt - 1) y_n - y_{n-1}/dtt;  u = (Sigma^T Sigma)^+ z
//   post:     j_n = y_n + Sigma u = P^LH y_n + P^S (y_n - y_{n-1})/dtt                (Eq. post_processing)
// Layouts (HBM): matrices row-major; vectors right-hand-side-major (R x N per slot); the ring
// holds y_{n-1} .. y_{n-K+1} in K-1 slots, slot = i mod (K-1); y_n overwrites the slot of
// y_{n-K+1} after the history sum has consumed it.
#include <cuda_bf16.h>

#include <cmath>
#include <algorithm>
#include <cstring>
#include <string>

#include "internal.h"
#include "umma.h"

namespace tdc {

struct Ctl {              // device-resident step state read by every kernel of a step
    int64_t n;            // current step (1-based)
    int64_t n0;           // step of the first output row of this tdcfie_step call
    void* out;            // currents_out of this call (nullptr: discard)
    int status;           // 0 ok, else TDCFIE_E_NONFINITE step recorded in bad_step
    int64_t bad_step;
};

struct StepPlan {
    int prec = TDCFIE_FP64;
    int R = 1, ne = 0, nc = 0, K = 0, nblk = 0, ring = 0;
    size_t esz = 8;
    void* blocks = nullptr;      // nblk x ne x ne (path precision): -A, alpha L2, -T_1 .. -T_{K-1}
    void* t0inv = nullptr;       // ne x ne
    void* pinv = nullptr;        // nc x nc
    void* E = nullptr;           // R x ne  (e_n)
    void* Hv = nullptr;          // R x ne  (h_n)
    void* ringbuf = nullptr;     // ring x R x ne
    void* b = nullptr;           // R x ne
    void* partial = nullptr;     // nblk x R x ne
    void* w = nullptr;           // R x ne
    void* z = nullptr;           // R x nc
    void* u = nullptr;           // R x nc
    const void** xptr = nullptr; // device array (unused for SIMT: computed in kernel)
    Ctl* ctl = nullptr;
    // rhs tables
    int* fn_ptr = nullptr; int* fn_tri = nullptr; double* fn_phi = nullptr;
    // bf16x3 path
    Bf16x3Gemm* gemm = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr;
    cudaEvent_t evA = nullptr, evB = nullptr;            // captured around the history sum
    cudaGraphNode_t nodeA = nullptr, nodeB = nullptr;    // their record nodes in the step graph
    std::vector<cudaEvent_t> hA, hB;                     // per-step events of a tdcfie_step call
    int launches_per_step = 0;
};

// ---------------------------------------------------------------- plane-wave tests
__constant__ double c7[7][4];
__constant__ double c3[3][4];

template <typename T>
__global__ void k_rhs(DevMesh m, const double* __restrict__ exc, int R, double dt, const Ctl* ctl,
                      const int* __restrict__ fn_ptr, const int* __restrict__ fn_tri, const double* __restrict__ fn_phi,
                      T* __restrict__ E, T* __restrict__ H) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= m.ne * R) return;
    const int r = idx / m.ne, mm = idx % m.ne;
    const double t = (double)ctl->n * dt;
    const double* P = exc + 11 * r;   // k(3) p(3) amp t0 width
    const double kx = P[0], ky = P[1], kz = P[2], px = P[3], py = P[4], pz = P[5];
    const double amp = P[6], t0 = P[7], wid = P[8];
    // h direction k x p
    const double hx = ky * pz - kz * py, hy = kz * px - kx * pz, hz = kx * py - ky * px;
    double e = 0.0;
    // the two triangles of edge mm: walk both supports through fn_* is for BC; RWG support from E table
    for (int side = 0; side < 2; ++side) {
        const int c = side == 0 ? m.cplus_[mm] : m.cminus_[mm];
        int j = 0;
        for (; j < 3; ++j) if (m.tedge[3 * c + j] == mm) break;
        const double* a = m.V + 3 * m.F[3 * c];
        const double* b = m.V + 3 * m.F[3 * c + 1];
        const double* cc = m.V + 3 * m.F[3 * c + 2];
        const double ex = b[0] - a[0], ey = b[1] - a[1], ez = b[2] - a[2];
        const double fx = cc[0] - a[0], fy = cc[1] - a[1], fz = cc[2] - a[2];
        const double nx = ey * fz - ez * fy, ny = ez * fx - ex * fz, nz = ex * fy - ey * fx;
        const double A = 0.5 * sqrt(nx * nx + ny * ny + nz * nz);
        const double* o = m.V + 3 * m.F[3 * c + j];
        const double s = m.tsign[3 * c + j] / (2.0 * A);
        for (int q = 0; q < 7; ++q) {
            const double x = c7[q][0] * a[0] + c7[q][1] * b[0] + c7[q][2] * cc[0];
            const double y = c7[q][0] * a[1] + c7[q][1] * b[1] + c7[q][2] * cc[1];
            const double zz = c7[q][0] * a[2] + c7[q][1] * b[2] + c7[q][2] * cc[2];
            const double arg = (t - (kx * x + ky * y + kz * zz) - t0) / wid;
            const double env = amp * exp(-arg * arg);
            e += c7[q][3] * A * env * s * ((x - o[0]) * px + (y - o[1]) * py + (zz - o[2]) * pz);
        }
    }
    double h = 0.0;
    for (int q2 = fn_ptr[mm]; q2 < fn_ptr[mm + 1]; ++q2) {
        const int ft = fn_tri[q2];
        const double* ph = fn_phi + 3 * q2;
        const double* w0 = m.fV + 3 * m.fF[3 * ft];
        const double* w1 = m.fV + 3 * m.fF[3 * ft + 1];
        const double* w2 = m.fV + 3 * m.fF[3 * ft + 2];
        const double ex = w1[0] - w0[0], ey = w1[1] - w0[1], ez = w1[2] - w0[2];
        const double fx = w2[0] - w0[0], fy = w2[1] - w0[1], fz = w2[2] - w0[2];
        const double nx = ey * fz - ez * fy, ny = ez * fx - ex * fz, nz = ex * fy - ey * fx;
        const double A = 0.5 * sqrt(nx * nx + ny * ny + nz * nz);
        const double* W[3] = {w0, w1, w2};
        for (int q = 0; q < 3; ++q) {
            const double x = c3[q][0] * w0[0] + c3[q][1] * w1[0] + c3[q][2] * w2[0];
            const double y = c3[q][0] * w0[1] + c3[q][1] * w1[1] + c3[q][2] * w2[1];
            const double zz = c3[q][0] * w0[2] + c3[q][1] * w1[2] + c3[q][2] * w2[2];
            double gx = 0, gy = 0, gz = 0;
            for (int j = 0; j < 3; ++j) {
                gx += ph[j] * (x - W[j][0]); gy += ph[j] * (y - W[j][1]); gz += ph[j] * (zz - W[j][2]);
            }
            const double arg = (t - (kx * x + ky * y + kz * zz) - t0) / wid;
            const double env = amp * exp(-arg * arg);
            h += c3[q][3] * A * env * (gx * hx + gy * hy + gz * hz) / (2.0 * A);
        }
    }
    E[(int64_t)r * m.ne + mm] = (T)e;
    H[(int64_t)r * m.ne + mm] = (T)h;
}

// ---------------------------------------------------------------- multi-block GEMV (SIMT)
// partial[q][r][i] = sum_j B_q[i][j] x_q[r][j] for one warp per (row i, block q); x_q is e_n, h_n
// or a ring slot chosen from the device step counter.
template <typename T> struct Vec2;
template <> struct Vec2<double> { using type = double2; };
template <> struct Vec2<float> { using type = float4; };

template <typename T, int RMAX>
__device__ __forceinline__ void warp_rows(const T* __restrict__ B, int ncols, const T* __restrict__ x, int R,
                                          int ldx, double* acc) {
    const int lane = threadIdx.x & 31;
    T s[RMAX];
#pragma unroll
    for (int r = 0; r < RMAX; ++r) s[r] = 0;
    for (int j = lane; j < ncols; j += 32) {
        const T a = B[j];
#pragma unroll
        for (int r = 0; r < RMAX; ++r)
            if (r < R) s[r] += a * x[(int64_t)r * ldx + j];
    }
#pragma unroll
    for (int r = 0; r < RMAX; ++r) {
        T v = s[r];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        acc[r] = (double)v;
    }
}

template <typename T, int RMAX>
__global__ void k_history(const T* __restrict__ blocks, int nblk, int ne, int R, int ring, const Ctl* ctl,
                          const T* __restrict__ E, const T* __restrict__ H, const T* __restrict__ ringbuf,
                          T* __restrict__ partial) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int q = blockIdx.y;
    if (warp >= ne) return;
    const int64_t n = ctl->n;
    const T* x;
    if (q == 0) x = E;
    else if (q == 1) x = H;
    else {
        const int64_t k = q - 1;                 // lag of this history block
        int64_t slot = (n - k) % ring;
        if (slot < 0) slot += ring;
        x = ringbuf + slot * (int64_t)R * ne;
    }
    double acc[RMAX];
    warp_rows<T, RMAX>(blocks + ((int64_t)q * ne + warp) * ne, ne, x, R, ne, acc);
    if ((threadIdx.x & 31) == 0)
        for (int r = 0; r < R; ++r) partial[((int64_t)q * R + r) * ne + warp] = (T)acc[r];
}

template <typename T>
__global__ void k_reduce(const T* __restrict__ partial, int nblk, int ne, int R, T* __restrict__ b) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ne * R) return;
    T s = 0;
    for (int q = 0; q < nblk; ++q) s += partial[(int64_t)q * R * ne + i];
    b[i] = s;
}

// y = M x for one square matrix, one warp per row; result to a ring slot or plain buffer
template <typename T, int RMAX>
__global__ void k_apply(const T* __restrict__ Mtx, int nrow, int ncol, int R, const T* __restrict__ x,
                        T* __restrict__ y, int ring, const Ctl* ctl) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (warp >= nrow) return;
    double acc[RMAX];
    warp_rows<T, RMAX>(Mtx + (int64_t)warp * ncol, ncol, x, R, ncol, acc);
    T* dst = y;
    if (ring > 0) dst = y + (ctl->n % ring) * (int64_t)R * nrow;
    if ((threadIdx.x & 31) == 0)
        for (int r = 0; r < R; ++r) dst[(int64_t)r * nrow + warp] = (T)acc[r];
}

// z[r][c] = sum_j tsign[c][j] w[r][tedge[c][j]],  w = (1/dtt - 1) y_n - y_{n-1}/dtt
template <typename T>
__global__ void k_project_in(DevMesh m, int R, int ring, const Ctl* ctl, const T* __restrict__ ringbuf, double dtt,
                             T* __restrict__ z) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= m.nc * R) return;
    const int r = idx / m.nc, c = idx % m.nc;
    const int64_t n = ctl->n;
    const T* yn = ringbuf + (n % ring) * (int64_t)R * m.ne + (int64_t)r * m.ne;
    const T* yp = ringbuf + ((n - 1) % ring) * (int64_t)R * m.ne + (int64_t)r * m.ne;
    const bool first = (n == 1);
    double s = 0.0;
    for (int j = 0; j < 3; ++j) {
        const int e = m.tedge[3 * c + j];
        const double w = (1.0 / dtt - 1.0) * (double)yn[e] - (first ? 0.0 : (double)yp[e]) / dtt;
        s += m.tsign[3 * c + j] * w;
    }
    z[(int64_t)r * m.nc + c] = (T)s;
}

// j[r][m] = y_n[r][m] + u[r][c+(m)] - u[r][c-(m)]; write to out, check finiteness
template <typename T>
__global__ void k_project_out(DevMesh m, int R, int ring, Ctl* ctl, const T* __restrict__ ringbuf,
                              const T* __restrict__ u) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= m.ne * R) return;
    const int r = idx / m.ne, e = idx % m.ne;
    const int64_t n = ctl->n;
    const T* yn = ringbuf + (n % ring) * (int64_t)R * m.ne + (int64_t)r * m.ne;
    const T val = yn[e] + u[(int64_t)r * m.nc + m.cplus_[e]] - u[(int64_t)r * m.nc + m.cminus_[e]];
    if (!isfinite((double)val) && atomicCAS(&ctl->status, 0, (int)TDCFIE_E_NONFINITE) == 0) ctl->bad_step = n;
    if (ctl->out) {
        T* o = reinterpret_cast<T*>(ctl->out);
        o[((n - ctl->n0) * R + r) * (int64_t)m.ne + e] = val;
    }
}

__global__ void k_advance(Ctl* ctl) { ctl->n += 1; }

// ---------------------------------------------------------------- plan construction
static size_t esize(int prec) { return prec == TDCFIE_FP64 ? 8 : 4; }

template <typename T>
static void launch_step(tdcfie_t h, StepPlan& p, cudaStream_t s) {
    const tdc::DevMesh& m = h->dm;
    const int R = p.R, ne = p.ne;
    const int tb = 256;
    k_rhs<T><<<(ne * R + tb - 1) / tb, tb, 0, s>>>(m, h->dexc, R, h->dt, p.ctl, p.fn_ptr, p.fn_tri, p.fn_phi,
                                                    (T*)p.E, (T*)p.Hv);
    const int wpb = 8;   // warps per block
    dim3 g((ne + wpb - 1) / wpb, p.nblk);
#define HIST(RM) k_history<T, RM><<<g, 32 * wpb, 0, s>>>((const T*)p.blocks, p.nblk, ne, R, p.ring, p.ctl, \
                                                           (const T*)p.E, (const T*)p.Hv, (const T*)p.ringbuf, (T*)p.partial)
#define APPLY(RM, M, nr, nc_, x, y, rg) k_apply<T, RM><<<((nr) + wpb - 1) / wpb, 32 * wpb, 0, s>>>((const T*)(M), nr, nc_, R, (const T*)(x), (T*)(y), rg, p.ctl)
    cudaEventRecord(p.evA, s);
    if (R == 1) HIST(1); else if (R <= 4) HIST(4); else HIST(8);
    k_reduce<T><<<(ne * R + tb - 1) / tb, tb, 0, s>>>((const T*)p.partial, p.nblk, ne, R, (T*)p.b);
    cudaEventRecord(p.evB, s);
    if (R == 1) APPLY(1, p.t0inv, ne, ne, p.b, p.ringbuf, p.ring);
    else if (R <= 4) APPLY(4, p.t0inv, ne, ne, p.b, p.ringbuf, p.ring);
    else APPLY(8, p.t0inv, ne, ne, p.b, p.ringbuf, p.ring);
    k_project_in<T><<<(p.nc * R + tb - 1) / tb, tb, 0, s>>>(m, R, p.ring, p.ctl, (const T*)p.ringbuf, h->dtt, (T*)p.z);
    if (R == 1) APPLY(1, p.pinv, p.nc, p.nc, p.z, p.u, 0);
    else if (R <= 4) APPLY(4, p.pinv, p.nc, p.nc, p.z, p.u, 0);
    else APPLY(8, p.pinv, p.nc, p.nc, p.z, p.u, 0);
    k_project_out<T><<<(ne * R + tb - 1) / tb, tb, 0, s>>>(m, R, p.ring, p.ctl, (const T*)p.ringbuf, (const T*)p.u);
    k_advance<<<1, 1, 0, s>>>(p.ctl);
#undef HIST
#undef APPLY
    p.launches_per_step = 8;
}

void free_plan(tdcfie_t h) {
    StepPlan* p = h->plan;
    if (!p) return;
    void* bufs[] = {p->blocks, p->t0inv, p->pinv, p->E, p->Hv, p->ringbuf, p->b, p->partial, p->w, p->z, p->u,
                    p->ctl, p->fn_ptr, p->fn_tri, p->fn_phi};
    for (void* b : bufs) if (b) cudaFree(b);
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->ev0) cudaEventDestroy(p->ev0);
    if (p->ev1) cudaEventDestroy(p->ev1);
    if (p->ev2) cudaEventDestroy(p->ev2);
    if (p->gemm) destroy_bf16x3(p->gemm);
    if (p->evA) cudaEventDestroy(p->evA);
    if (p->evB) cudaEventDestroy(p->evB);
    for (auto e : p->hA) cudaEventDestroy(e);
    for (auto e : p->hB) cudaEventDestroy(e);
    delete p;
    h->plan = nullptr;
}

#define CK(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) return cuda_fail(h, e_, #x); } while (0)

static void to_path(cudaStream_t s, int prec, const double* src, void* dst, int64_t n) {
    if (prec == TDCFIE_FP64) cudaMemcpyAsync(dst, src, n * 8, cudaMemcpyDeviceToDevice, s);
    else cast_f64_f32(s, src, (float*)dst, n);
}

tdcfie_status build_plan(tdcfie_t h) {
    free_plan(h);
    StepPlan* p = new StepPlan();
    h->plan = p;
    cudaStream_t s = h->stream;
    const tdc::Mesh& M = h->mesh;
    p->prec = h->opts.precision;
    p->R = (int)h->R;
    p->ne = M.ne; p->nc = M.nc; p->K = h->K;
    p->nblk = h->K + 1;              // -A, alpha L2, -T_1..-T_{K-1}
    p->ring = h->K - 1;
    p->esz = esize(p->prec);
    const int64_t ne = M.ne, nc = M.nc, R = p->R;
    if (p->prec == TDCFIE_BF16X3) {
        // the tensor-core path keeps FP32 vectors and splits matrices into bf16 hi/lo
        p->esz = 4;
    }
    const size_t es = p->esz;
    // rhs constant tables
    {
        const double s15 = std::sqrt(15.0);
        const double a1 = (9.0 - 2.0 * s15) / 21.0, b1 = (6.0 + s15) / 21.0, w1 = (155.0 + s15) / 1200.0;
        const double a2 = (9.0 + 2.0 * s15) / 21.0, b2 = (6.0 - s15) / 21.0, w2 = (155.0 - s15) / 1200.0;
        double r7[7][4] = {{1.0 / 3, 1.0 / 3, 1.0 / 3, 9.0 / 40.0}, {a1, b1, b1, w1}, {b1, a1, b1, w1}, {b1, b1, a1, w1},
                           {a2, b2, b2, w2}, {b2, a2, b2, w2}, {b2, b2, a2, w2}};
        double r3[3][4] = {{2.0 / 3, 1.0 / 6, 1.0 / 6, 1.0 / 3}, {1.0 / 6, 2.0 / 3, 1.0 / 6, 1.0 / 3},
                           {1.0 / 6, 1.0 / 6, 2.0 / 3, 1.0 / 3}};
        CK(cudaMemcpyToSymbolAsync(c7, r7, sizeof(r7), 0, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyToSymbolAsync(c3, r3, sizeof(r3), 0, cudaMemcpyHostToDevice, s));
        // BC functions by function: (fine triangle, 3 fluxes)
        std::vector<int> cnt(ne + 1, 0);
        for (size_t e = 0; e < M.bc_fn.size(); ++e) cnt[M.bc_fn[e] + 1]++;
        for (int64_t i = 0; i < ne; ++i) cnt[i + 1] += cnt[i];
        std::vector<int> tri(M.bc_fn.size());
        std::vector<double> ph(3 * M.bc_fn.size());
        std::vector<int> fill(cnt.begin(), cnt.end() - 1);
        for (int t = 0; t < M.nf; ++t)
            for (int e = M.bc_ptr[t]; e < M.bc_ptr[t + 1]; ++e) {
                const int pos = fill[M.bc_fn[e]]++;
                tri[pos] = t;
                for (int k = 0; k < 3; ++k) ph[3 * pos + k] = M.bc_phi[3 * e + k];
            }
        CK(cudaMalloc(&p->fn_ptr, sizeof(int) * (ne + 1)));
        CK(cudaMalloc(&p->fn_tri, sizeof(int) * tri.size()));
        CK(cudaMalloc(&p->fn_phi, sizeof(double) * ph.size()));
        CK(cudaMemcpyAsync(p->fn_ptr, cnt.data(), sizeof(int) * (ne + 1), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(p->fn_tri, tri.data(), sizeof(int) * tri.size(), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(p->fn_phi, ph.data(), sizeof(double) * ph.size(), cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));
    }
    CK(cudaMalloc(&p->ctl, sizeof(Ctl)));
    CK(cudaMalloc(&p->E, es * R * ne));
    CK(cudaMalloc(&p->Hv, es * R * ne));
    CK(cudaMalloc(&p->ringbuf, es * p->ring * R * ne));
    CK(cudaMalloc(&p->b, es * R * ne));
    CK(cudaMalloc(&p->partial, es * p->nblk * R * ne));
    CK(cudaMalloc(&p->z, es * R * nc));
    CK(cudaMalloc(&p->u, es * R * nc));
    if (p->prec == TDCFIE_BF16X3) {
        tdcfie_status st = build_bf16x3(h, p);
        if (st != TDCFIE_OK) return st;
    } else {
        CK(cudaMalloc(&p->blocks, es * p->nblk * ne * ne));
        CK(cudaMalloc(&p->t0inv, es * ne * ne));
        CK(cudaMalloc(&p->pinv, es * nc * nc));
        // block 0: -A, block 1: alpha L2, block 1+k: -T_k
        double* tmp = nullptr;
        CK(cudaMalloc(&tmp, 8 * ne * ne));
        CK(cudaMemcpyAsync(tmp, h->A, 8 * ne * ne, cudaMemcpyDeviceToDevice, s));
        axpby(s, ne * ne, 0.0, tmp, -1.0, tmp);
        to_path(s, p->prec, tmp, p->blocks, ne * ne);
        CK(cudaMemcpyAsync(tmp, h->L2, 8 * ne * ne, cudaMemcpyDeviceToDevice, s));
        axpby(s, ne * ne, 0.0, tmp, h->alpha, tmp);
        to_path(s, p->prec, tmp, (char*)p->blocks + es * ne * ne, ne * ne);
        for (int k = 1; k < h->K; ++k) {
            CK(cudaMemcpyAsync(tmp, h->T + (int64_t)k * ne * ne, 8 * ne * ne, cudaMemcpyDeviceToDevice, s));
            axpby(s, ne * ne, 0.0, tmp, -1.0, tmp);
            to_path(s, p->prec, tmp, (char*)p->blocks + es * (1 + k) * ne * ne, ne * ne);
        }
        to_path(s, p->prec, h->T0inv, p->t0inv, ne * ne);
        to_path(s, p->prec, h->PinvS, p->pinv, nc * nc);
        CK(cudaStreamSynchronize(s));
        cudaFree(tmp);
    }
    CK(cudaEventCreate(&p->ev0));
    CK(cudaEventCreate(&p->ev1));
    CK(cudaEventCreate(&p->ev2));
    CK(cudaEventCreate(&p->evA));
    CK(cudaEventCreate(&p->evB));
    h->hist_bytes = (double)p->nblk * ne * ne * (p->prec == TDCFIE_FP64 ? 8.0 : 4.0);
    return plan_reset(h);
}

tdcfie_status plan_reset(tdcfie_t h) {
    StepPlan* p = h->plan;
    cudaStream_t s = h->stream;
    Ctl c{1, 1, nullptr, 0, 0};
    CK(cudaMemcpyAsync(p->ctl, &c, sizeof(Ctl), cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(p->ringbuf, 0, p->esz * p->ring * p->R * p->ne, s));
    CK(cudaStreamSynchronize(s));
    return TDCFIE_OK;
}

tdcfie_status plan_step(tdcfie_t h, int64_t nsteps, void* out) {
    StepPlan* p = h->plan;
    cudaStream_t s = h->stream;
    if (h->own_stream) {
        // outputs may come from work queued on the caller's legacy default stream
        CK(cudaEventRecord(h->ev_in, 0));
        CK(cudaStreamWaitEvent(s, h->ev_in, 0));
    }
    if (!p->exec) {
        // capture one step
        CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        if (p->prec == TDCFIE_FP64) launch_step<double>(h, *p, s);
        else if (p->prec == TDCFIE_FP32) launch_step<float>(h, *p, s);
        else launch_step_bf16x3(h, p, s);
        CK(cudaStreamEndCapture(s, &p->graph));
        CK(cudaGraphInstantiate(&p->exec, p->graph, 0));
        size_t nn = 0;
        CK(cudaGraphGetNodes(p->graph, nullptr, &nn));
        std::vector<cudaGraphNode_t> nodes(nn);
        CK(cudaGraphGetNodes(p->graph, nodes.data(), &nn));
        for (auto nd : nodes) {
            cudaGraphNodeType ty;
            CK(cudaGraphNodeGetType(nd, &ty));
            if (ty != cudaGraphNodeTypeEventRecord) continue;
            cudaEvent_t ev;
            CK(cudaGraphEventRecordNodeGetEvent(nd, &ev));
            if (ev == p->evA) p->nodeA = nd;
            if (ev == p->evB) p->nodeB = nd;
        }
    }
    // per-step events around the history sum (rotated into the executable graph before each launch)
    const int64_t nev = std::min<int64_t>(nsteps, 4096);
    while ((int64_t)p->hA.size() < nev) {
        cudaEvent_t a, b;
        CK(cudaEventCreate(&a));
        CK(cudaEventCreate(&b));
        p->hA.push_back(a);
        p->hB.push_back(b);
    }
    // set the output base of this call: n0 = current n
    Ctl c;
    CK(cudaMemcpyAsync(&c, p->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    c.n0 = c.n;
    c.out = out;
    CK(cudaMemcpyAsync(p->ctl, &c, sizeof(Ctl), cudaMemcpyHostToDevice, s));
    CK(cudaEventRecord(p->ev0, s));
    for (int64_t i = 0; i < nsteps; ++i) {
        if (i < nev && p->nodeA && p->nodeB) {
            CK(cudaGraphExecEventRecordNodeSetEvent(p->exec, p->nodeA, p->hA[i]));
            CK(cudaGraphExecEventRecordNodeSetEvent(p->exec, p->nodeB, p->hB[i]));
        }
        CK(cudaGraphLaunch(p->exec, s));
    }
    CK(cudaEventRecord(p->ev1, s));
    CK(cudaMemcpyAsync(&c, p->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, p->ev0, p->ev1);
    h->last_step_ms = ms / (nsteps > 0 ? nsteps : 1);
    double hs = 0.0;
    int64_t cnt = 0;
    for (int64_t i = 0; i < nev && p->nodeA && p->nodeB; ++i) {
        float e = 0.f;
        if (cudaEventElapsedTime(&e, p->hA[i], p->hB[i]) == cudaSuccess) { hs += e; ++cnt; }
    }
    h->last_hist_ms = cnt ? hs / cnt : 0.0;
    h->last_launches = nsteps * p->launches_per_step;
    if (c.status != 0)
        return fail(h, TDCFIE_E_NONFINITE, "non-finite current at step " + std::to_string(c.bad_step));
    return TDCFIE_OK;
}

}  // namespace tdc
