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
#include "gmres.h"
#include "simt.h"
#include "plan.h"
#include "umma.h"

namespace tdc {

// ---------------------------------------------------------------- plane-wave tests
// e_m(t_n), h_m(t_n) for every (edge, wave), waves fastest (a warp shares one edge's points)
template <typename T>
__global__ void k_rhs(int ne, const double* __restrict__ exc, int R, double dt, const Ctl* ctl,
                      const int* __restrict__ pptr, const T* __restrict__ px, const T* __restrict__ pc,
                      const int* __restrict__ nE, T* __restrict__ E, T* __restrict__ H) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= ne * R) return;
    const int r = idx % R, mm = idx / R;
    T e, h;
    rhs_edge<T>(exc + 11 * r, ctl->n, dt, mm, pptr, px, pc, nE, e, h);
    E[(int64_t)r * ne + mm] = e;
    H[(int64_t)r * ne + mm] = h;
}

// Per-block partial sums of the history, kept in FP64 for every path precision
template <typename T, int RMAX>
__global__ void k_history(const T* __restrict__ blocks, int nblk, int ne, int R, int ring, const Ctl* ctl,
                          const T* __restrict__ E, const T* __restrict__ H, const T* __restrict__ ringbuf,
                          double* __restrict__ partial) {
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
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int r = 0; r < RMAX; ++r)
            if (r < R) partial[((int64_t)q * R + r) * ne + warp] = acc[r];
    }
}

// FP32 history for several right-hand sides: one warp per ROWS rows, so that each lane's loads of
// the R history vectors serve ROWS rows; error-free accumulation as in RowDot<float>
template <int RMAX, int ROWS>
__global__ void __launch_bounds__(256) k_history_rows(const float* __restrict__ blocks, int ne, int R, int ring,
                                                      const Ctl* ctl, const float* __restrict__ E,
                                                      const float* __restrict__ H, const float* __restrict__ ringbuf,
                                                      double* __restrict__ partial) {
    const int row0 = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * ROWS;
    const int q = blockIdx.y;
    if (row0 >= ne) return;
    const int lane = threadIdx.x & 31;
    const int64_t n = ctl->n;
    const float* x;
    if (q == 0) x = E;
    else if (q == 1) x = H;
    else {
        int64_t slot = (n - (q - 1)) % ring;
        if (slot < 0) slot += ring;
        x = ringbuf + slot * (int64_t)R * ne;
    }
    const float* Bq = blocks + (int64_t)q * ne * ne;
    float hi[ROWS][RMAX], lo[ROWS][RMAX];
#pragma unroll
    for (int i = 0; i < ROWS; ++i)
#pragma unroll
        for (int r = 0; r < RMAX; ++r) hi[i][r] = lo[i][r] = 0.f;
    if ((ne & 3) == 0) {     // rows and vectors start on 16-byte boundaries
        for (int j = lane; j < (ne >> 2); j += 32) {
            float4 xv[RMAX];
#pragma unroll
            for (int r = 0; r < RMAX; ++r)
                if (r < R) xv[r] = reinterpret_cast<const float4*>(x + (int64_t)r * ne)[j];
#pragma unroll
            for (int i = 0; i < ROWS; ++i) {
                if (row0 + i >= ne) break;
                const float4 a = reinterpret_cast<const float4*>(Bq + (int64_t)(row0 + i) * ne)[j];
#pragma unroll
                for (int r = 0; r < RMAX; ++r)
                    if (r < R) {
                        ff_add(hi[i][r], lo[i][r], a.x, xv[r].x);
                        ff_add(hi[i][r], lo[i][r], a.y, xv[r].y);
                        ff_add(hi[i][r], lo[i][r], a.z, xv[r].z);
                        ff_add(hi[i][r], lo[i][r], a.w, xv[r].w);
                    }
            }
        }
    } else {
        for (int j = lane; j < ne; j += 32) {
            float xv[RMAX];
#pragma unroll
            for (int r = 0; r < RMAX; ++r)
                if (r < R) xv[r] = x[(int64_t)r * ne + j];
#pragma unroll
            for (int i = 0; i < ROWS; ++i) {
                if (row0 + i >= ne) break;
                const float a = Bq[(int64_t)(row0 + i) * ne + j];
#pragma unroll
                for (int r = 0; r < RMAX; ++r)
                    if (r < R) ff_add(hi[i][r], lo[i][r], a, xv[r]);
            }
        }
    }
#pragma unroll
    for (int i = 0; i < ROWS; ++i)
#pragma unroll
        for (int r = 0; r < RMAX; ++r) {
            double v = (double)hi[i][r] + (double)lo[i][r];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0 && r < R && row0 + i < ne) partial[((int64_t)q * R + r) * ne + row0 + i] = v;
        }
}

template <typename T>
__global__ void k_reduce(const double* __restrict__ partial, int nblk, int ne, int R, T* __restrict__ b) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ne * R) return;
    double s = 0;
    for (int q = 0; q < nblk; ++q) s += partial[(int64_t)q * R * ne + i];
    b[i] = (T)s;
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
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int r = 0; r < RMAX; ++r)
            if (r < R) dst[(int64_t)r * nrow + warp] = (T)acc[r];
    }
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
    z[(int64_t)r * m.nc + c] = (T)project_in_value<T>(m, c, yn, yp, n == 1, dtt);
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
    if (ctl->yout) {
        T* o = reinterpret_cast<T*>(ctl->yout);
        o[((n - ctl->n0) * R + r) * (int64_t)m.ne + e] = yn[e];
    }
}

__global__ void k_advance(Ctl* ctl) { ctl->n += 1; }

// ---------------------------------------------------------------- plan construction
static size_t esize(int prec) { return prec == TDCFIE_FP64 ? 8 : 4; }

template <typename T>
void launch_rhs(tdcfie_t h, StepPlan& p, cudaStream_t s) {
    const int tb = 256;
    k_rhs<T><<<(p.ne * p.R + tb - 1) / tb, tb, 0, s>>>(p.ne, h->dexc, p.R, h->dt, p.ctl, p.pptr, (const T*)p.px,
                                                        (const T*)p.pc, p.pnE, (T*)p.E, (T*)p.Hv);
}
template void launch_rhs<double>(tdcfie_t, StepPlan&, cudaStream_t);
template void launch_rhs<float>(tdcfie_t, StepPlan&, cudaStream_t);

template <typename T>
static cudaError_t launch_step(tdcfie_t h, StepPlan& p, cudaStream_t s) {
    if (p.fact) return launch_step_fact<T>(h, p, s);
    const tdc::DevMesh& m = h->dm;
    const int R = p.R, ne = p.ne;
    const int tb = 256;
    launch_rhs<T>(h, p, s);
    const int wpb = 8;   // warps per block
    dim3 g((ne + wpb - 1) / wpb, p.nblk);
#define HIST(RM) k_history<T, RM><<<g, 32 * wpb, 0, s>>>((const T*)p.blocks, p.nblk, ne, R, p.ring, p.ctl, \
                                                           (const T*)p.E, (const T*)p.Hv, (const T*)p.ringbuf, (double*)p.partial)
#define APPLY(RM, M, nr, nc_, x, y, rg) k_apply<T, RM><<<((nr) + wpb - 1) / wpb, 32 * wpb, 0, s>>>((const T*)(M), nr, nc_, R, (const T*)(x), (T*)(y), rg, p.ctl)
    cudaEventRecordWithFlags(p.evA, s, cudaEventRecordExternal);
    if (R == 1 || sizeof(T) == 8) {
        if (R == 1) HIST(1); else if (R <= 4) HIST(4); else HIST(8);
    } else {
        // FP32 with several waves: 4 rows per warp up to 4 waves, 2 rows (fewer registers) above
#define HISTR(RM, ROWS) k_history_rows<RM, ROWS><<<dim3((ne + wpb * ROWS - 1) / (wpb * ROWS), p.nblk), 32 * wpb, 0, s>>>( \
            (const float*)p.blocks, ne, R, p.ring, p.ctl, (const float*)p.E, (const float*)p.Hv,                       \
            (const float*)p.ringbuf, (double*)p.partial)
        if (R <= 4) HISTR(4, 4); else HISTR(8, 2);
#undef HISTR
    }
    k_reduce<T><<<(ne * R + tb - 1) / tb, tb, 0, s>>>((const double*)p.partial, p.nblk, ne, R, (T*)p.b);
    cudaEventRecordWithFlags(p.evB, s, cudaEventRecordExternal);
    p.launches_per_step = 0;
    if (p.mlp_on) launch_mlp_guess<T>(&p, s);
    if (p.gmres_on) {
        const cudaError_t e = launch_gmres<T>(h, &p, (const T*)p.b, (const T*)p.guessbuf, (const T*)p.t0mat,
                                              (T*)p.ringbuf, s);
        if (e != cudaSuccess) return e;
    } else if (R == 1) APPLY(1, p.t0inv, ne, ne, p.b, p.ringbuf, p.ring);
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
    p.launches_per_step += 8 - (p.gmres_on ? 1 : 0);
    return cudaGetLastError();
}

tdcfie_status plan_gmres_stats(tdcfie_t h, long long* out6) {
    StepPlan* p = h->plan;
    if (!p || !p->gm) return fail(h, TDCFIE_E_STATE, "GMRES solver not active on this handle");
    const cudaError_t e = gmres_stats(p->gm, out6);
    if (e != cudaSuccess) return cuda_fail(h, e, "gmres_stats");
    return TDCFIE_OK;
}

void free_plan(tdcfie_t h) {
    StepPlan* p = h->plan;
    if (!p) return;
    void* bufs[] = {p->blocks, p->t0inv, p->pinv, p->E, p->Hv, p->ringbuf, p->b, p->partial, p->w, p->z, p->u,
                    p->ctl, p->pptr, p->pnE, p->px, p->pc};
    for (void* b : bufs) if (b) cudaFree(b);
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->ev0) cudaEventDestroy(p->ev0);
    if (p->ev1) cudaEventDestroy(p->ev1);
    if (p->ev2) cudaEventDestroy(p->ev2);
    if (p->gemm) destroy_tc(p->gemm);
    if (p->gm) destroy_gmres(p->gm);
    if (p->mlp) destroy_mlp(p->mlp);
    if (p->fact) destroy_fact(p->fact);
    if (p->t0mat) cudaFree(p->t0mat);
    if (p->guessbuf) cudaFree(p->guessbuf);
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
    const bool tensor = p->prec == TDCFIE_BF16X3 || p->prec == TDCFIE_FP16X3;
    if (h->formulation != TDCFIE_FORMULATION_QHP_CFIE && (tensor || h->history_form != TDCFIE_HISTORY_DENSE))
        return fail(h, TDCFIE_E_UNSUPPORTED, "the comparison formulation runs on the dense FP64 and FP32 paths");
    if (tensor) p->esz = 4;   // the tensor-core paths keep FP32 vectors, 16-bit hi/lo matrices
    const size_t es = p->esz;
    // rhs quadrature tables (host, FP64), uploaded in the path precision
    {
        const double s15 = std::sqrt(15.0);
        const double a1 = (9.0 - 2.0 * s15) / 21.0, b1 = (6.0 + s15) / 21.0, w1 = (155.0 + s15) / 1200.0;
        const double a2 = (9.0 + 2.0 * s15) / 21.0, b2 = (6.0 - s15) / 21.0, w2 = (155.0 - s15) / 1200.0;
        const double r7[7][4] = {{1.0 / 3, 1.0 / 3, 1.0 / 3, 9.0 / 40.0}, {a1, b1, b1, w1}, {b1, a1, b1, w1},
                                 {b1, b1, a1, w1}, {a2, b2, b2, w2}, {b2, a2, b2, w2}, {b2, b2, a2, w2}};
        const double r3[3][4] = {{2.0 / 3, 1.0 / 6, 1.0 / 6, 1.0 / 3}, {1.0 / 6, 2.0 / 3, 1.0 / 6, 1.0 / 3},
                                 {1.0 / 6, 1.0 / 6, 2.0 / 3, 1.0 / 3}};
        std::vector<std::vector<double>> pts(ne), cfs(ne);
        std::vector<int> nE(ne, 0);
        auto area = [](const double* a, const double* b, const double* c) {
            const double ex = b[0] - a[0], ey = b[1] - a[1], ez = b[2] - a[2];
            const double fx = c[0] - a[0], fy = c[1] - a[1], fz = c[2] - a[2];
            const double nx = ey * fz - ez * fy, ny = ez * fx - ex * fz, nz = ex * fy - ey * fx;
            return 0.5 * std::sqrt(nx * nx + ny * ny + nz * nz);
        };
        for (int c = 0; c < M.nc; ++c) {
            const double* v[3] = {&M.V[3 * M.F[3 * c]], &M.V[3 * M.F[3 * c + 1]], &M.V[3 * M.F[3 * c + 2]]};
            const double A = area(v[0], v[1], v[2]);
            for (int j = 0; j < 3; ++j) {
                const int m = M.tedge[3 * c + j];
                const double sgn = M.tsign[3 * c + j] / (2.0 * A);
                for (int q = 0; q < 7; ++q) {
                    double x[3];
                    for (int k = 0; k < 3; ++k) x[k] = r7[q][0] * v[0][k] + r7[q][1] * v[1][k] + r7[q][2] * v[2][k];
                    for (int k = 0; k < 3; ++k) {
                        pts[m].push_back(x[k]);
                        cfs[m].push_back(r7[q][3] * A * sgn * (x[k] - v[j][k]));
                    }
                    nE[m]++;
                }
            }
        }
        for (int t = 0; t < M.nf; ++t) {
            const double* v[3] = {&M.fV[3 * M.fF[3 * t]], &M.fV[3 * M.fF[3 * t + 1]], &M.fV[3 * M.fF[3 * t + 2]]};
            const double A = area(v[0], v[1], v[2]);
            for (int e = M.bc_ptr[t]; e < M.bc_ptr[t + 1]; ++e) {
                const int m = M.bc_fn[e];
                const double* ph = &M.bc_phi[3 * e];
                for (int q = 0; q < 3; ++q) {
                    double x[3];
                    for (int k = 0; k < 3; ++k) x[k] = r3[q][0] * v[0][k] + r3[q][1] * v[1][k] + r3[q][2] * v[2][k];
                    for (int k = 0; k < 3; ++k) {
                        pts[m].push_back(x[k]);
                        double g = 0.0;
                        for (int j = 0; j < 3; ++j) g += ph[j] * (x[k] - v[j][k]);
                        cfs[m].push_back(r3[q][3] * A * g / (2.0 * A));
                    }
                }
            }
        }
        // e-points were pushed before any h-point of the same edge only if all coarse passes ran
        // first, which they did (coarse loop precedes fine loop)
        std::vector<int> ptr(ne + 1, 0);
        for (int64_t m = 0; m < ne; ++m) ptr[m + 1] = ptr[m] + (int)(pts[m].size() / 3);
        std::vector<double> X(3 * (size_t)ptr[ne]), C(3 * (size_t)ptr[ne]);
        for (int64_t m = 0; m < ne; ++m) {
            std::copy(pts[m].begin(), pts[m].end(), X.begin() + 3 * ptr[m]);
            std::copy(cfs[m].begin(), cfs[m].end(), C.begin() + 3 * ptr[m]);
        }
        const size_t pes = (p->prec == TDCFIE_FP64) ? 8 : 4;
        CK(cudaMalloc(&p->pptr, sizeof(int) * (ne + 1)));
        CK(cudaMalloc(&p->pnE, sizeof(int) * ne));
        CK(cudaMalloc(&p->px, pes * X.size()));
        CK(cudaMalloc(&p->pc, pes * C.size()));
        CK(cudaMemcpy(p->pptr, ptr.data(), sizeof(int) * (ne + 1), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(p->pnE, nE.data(), sizeof(int) * ne, cudaMemcpyHostToDevice));
        if (pes == 8) {
            CK(cudaMemcpy(p->px, X.data(), 8 * X.size(), cudaMemcpyHostToDevice));
            CK(cudaMemcpy(p->pc, C.data(), 8 * C.size(), cudaMemcpyHostToDevice));
        } else {
            std::vector<float> Xf(X.begin(), X.end()), Cf(C.begin(), C.end());
            CK(cudaMemcpy(p->px, Xf.data(), 4 * Xf.size(), cudaMemcpyHostToDevice));
            CK(cudaMemcpy(p->pc, Cf.data(), 4 * Cf.size(), cudaMemcpyHostToDevice));
        }
    }
    CK(cudaMalloc(&p->ctl, sizeof(Ctl)));
    CK(cudaMalloc(&p->E, es * R * ne));
    CK(cudaMalloc(&p->Hv, es * R * ne));
    CK(cudaMalloc(&p->ringbuf, es * p->ring * R * ne));
    CK(cudaMalloc(&p->b, es * R * ne));
    CK(cudaMalloc(&p->partial, sizeof(double) * p->nblk * R * ne));
    CK(cudaMalloc(&p->z, es * R * nc));
    CK(cudaMalloc(&p->u, es * R * nc));
    if (tensor) {
        tdcfie_status st = build_tc(h, p);
        if (st != TDCFIE_OK) return st;
    } else if (h->formulation == TDCFIE_FORMULATION_MFIE) {
        // mixed TD-MFIE (a comparison formulation of Sec. V): sum_k MM'_k j_{n-k} = h_n with
        // MM'_0 = MM_0 + G/2; block 0 (e) zero, block 1 (h) the identity, block 1+k: -MM_k; the
        // unknown is j itself, so the projector product is zero and the post-processing returns y
        CK(cudaMalloc(&p->blocks, es * p->nblk * ne * ne));
        CK(cudaMalloc(&p->t0inv, es * ne * ne));
        CK(cudaMalloc(&p->pinv, es * nc * nc));
        CK(cudaMemsetAsync(p->blocks, 0, es * ne * ne, s));
        CK(cudaMemsetAsync(p->pinv, 0, es * nc * nc, s));
        double *tmp = nullptr, *work = nullptr;
        CK(cudaMalloc(&tmp, 8 * ne * ne));
        CK(cudaMalloc(&work, 8 * (2 * ne + 2)));
        fill_identity(s, tmp, (int)ne, 1.0);
        to_path(s, p->prec, tmp, (char*)p->blocks + es * ne * ne, ne * ne);
        for (int k = 1; k < h->K; ++k) {
            CK(cudaMemcpyAsync(tmp, h->MM + (int64_t)k * ne * ne, 8 * ne * ne, cudaMemcpyDeviceToDevice, s));
            axpby(s, ne * ne, 0.0, tmp, -1.0, tmp);
            to_path(s, p->prec, tmp, (char*)p->blocks + es * (1 + k) * ne * ne, ne * ne);
        }
        CK(cudaMemcpyAsync(tmp, h->MM, 8 * ne * ne, cudaMemcpyDeviceToDevice, s));
        axpby(s, ne * ne, 0.5, h->G, 1.0, tmp);
        const int singular = invert(s, tmp, (int)ne, work);
        to_path(s, p->prec, tmp, p->t0inv, ne * ne);
        CK(cudaStreamSynchronize(s));
        cudaFree(tmp);
        cudaFree(work);
        if (singular) return fail(h, TDCFIE_E_STATE, "G/2 + MM_0 is singular");
    } else if (h->history_form == TDCFIE_HISTORY_FACTORED) {
        tdcfie_status st = build_fact(h, p);
        if (st != TDCFIE_OK) return st;
        h->step_bytes = fact_step_bytes(p);
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
    if (!tensor && !p->fact) {
        h->hist_bytes = (double)p->nblk * ne * ne * es;
        h->step_bytes = h->hist_bytes + (double)ne * ne * es + (double)nc * nc * es;
    }
    if (h->opts.solver == TDCFIE_SOLVE_GMRES) {
        const tdcfie_status st = plan_set_solver(h, h->opts.solver, h->opts.guess, h->opts.gmres_tol);
        if (st != TDCFIE_OK) return st;
    }
    return plan_reset(h);
}

// Select the per-step solve of an existing plan; GMRES state, T_0 in the path precision and the
// learned-guess network are allocated on first use.  The step graph is captured again at the next
// step.
tdcfie_status plan_set_solver(tdcfie_t h, int solver, int guess, double tol) {
    StepPlan* p = h->plan;
    cudaStream_t s = h->stream;
    const int64_t ne = p->ne, R = p->R;
    const size_t es = p->esz;
    if (solver == TDCFIE_SOLVE_GMRES && (p->prec == TDCFIE_BF16X3 || p->prec == TDCFIE_FP16X3))
        return fail(h, TDCFIE_E_UNSUPPORTED, "GMRES runs on the FP64 and FP32 paths");
    if (solver == TDCFIE_SOLVE_GMRES && p->fact)
        return fail(h, TDCFIE_E_UNSUPPORTED, "the factored history form uses the direct solve");
    if (solver == TDCFIE_SOLVE_GMRES && h->formulation != TDCFIE_FORMULATION_QHP_CFIE)
        return fail(h, TDCFIE_E_UNSUPPORTED, "the comparison formulation uses the direct solve");
    const bool learned = guess == TDCFIE_GUESS_MLP || guess == TDCFIE_GUESS_MLP_EXTRAP;
    if (solver == TDCFIE_SOLVE_GMRES && guess == TDCFIE_GUESS_EXTRAP && p->ring < 4)
        return fail(h, TDCFIE_E_UNSUPPORTED, "the extrapolated guess needs K - 1 >= 4 stored steps");
    if (solver == TDCFIE_SOLVE_GMRES && learned && p->ring < 8)
        return fail(h, TDCFIE_E_UNSUPPORTED, "the learned guess needs K - 1 >= 8 stored steps");
    h->opts.solver = solver;
    h->opts.guess = guess;
    h->opts.gmres_tol = tol;
    if (solver == TDCFIE_SOLVE_GMRES) {
        if (!p->t0mat) {
            CK(cudaMalloc(&p->t0mat, es * ne * ne));
            to_path(s, p->prec, h->T, p->t0mat, ne * ne);
            CK(cudaMalloc(&p->guessbuf, es * R * ne));
            CK(cudaMemsetAsync(p->guessbuf, 0, es * R * ne, s));
            CK(cudaStreamSynchronize(s));
        }
        if (!p->gm) CK(build_gmres(h, p));
        gmres_set_tol(p->gm, tol);
        if (learned && !p->mlp) CK(build_mlp(p));
    }
    p->gmres_on = solver == TDCFIE_SOLVE_GMRES;
    p->mlp_on = p->gmres_on && learned;
    p->guess_extrap = guess == TDCFIE_GUESS_MLP_EXTRAP;
    if (p->exec) { cudaGraphExecDestroy(p->exec); p->exec = nullptr; }
    if (p->graph) { cudaGraphDestroy(p->graph); p->graph = nullptr; }
    p->nodeA = p->nodeB = nullptr;
    return TDCFIE_OK;
}

tdcfie_status plan_reset(tdcfie_t h) {
    StepPlan* p = h->plan;
    cudaStream_t s = h->stream;
    Ctl c{1, 1, nullptr, 0, 0, 0, nullptr};
    if (p->gm) CK(reset_gmres_stats(p->gm));
    CK(cudaMemcpyAsync(p->ctl, &c, sizeof(Ctl), cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(p->ringbuf, 0, p->esz * p->ring * p->R * p->ne, s));
    if (p->fact) {
        const tdcfie_status st = reset_fact(h, p);
        if (st != TDCFIE_OK) return st;
    }
    if (p->gemm) CK(reset_tc(p->gemm, p->ring, p->ne, s));
    CK(cudaStreamSynchronize(s));
    return TDCFIE_OK;
}

// Enqueue one step of h on s (s must be capturing a graph).
cudaError_t capture_step(tdcfie_t h, cudaStream_t s) {
    StepPlan* p = h->plan;
    if (p->prec == TDCFIE_FP64) return launch_step<double>(h, *p, s);
    if (p->prec == TDCFIE_FP32) return launch_step<float>(h, *p, s);
    launch_step_tc(h, p, s);
    return cudaGetLastError();
}

// Output base of the next steps of h (synchronous on h's stream): step n writes row n - n0.
tdcfie_status plan_set_outputs(tdcfie_t h, void* out, void* yout) {
    StepPlan* p = h->plan;
    cudaStream_t s = h->stream;
    Ctl c;
    CK(cudaMemcpyAsync(&c, p->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    c.n0 = c.n;
    c.out = out;
    c.yout = yout;
    CK(cudaMemcpyAsync(p->ctl, &c, sizeof(Ctl), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    return TDCFIE_OK;
}

// Status of the step state words: device timeout, then a non-finite current, then a GMRES solve that
// stopped above its tolerance (each with the first step it happened at)
static tdcfie_status status_of(tdcfie_t h, const Ctl& c) {
    if (c.timeout)
        return fail(h, TDCFIE_E_TIMEOUT, "a bounded device-side wait ran out (tensor-core pipeline)");
    if (c.status != 0)
        return fail(h, TDCFIE_E_NONFINITE, "non-finite current at step " + std::to_string(c.bad_step));
    if (c.noconv)
        return fail(h, TDCFIE_E_NOCONV, "GMRES stopped above gmres_tol (gmres_maxit reached) at step " +
                                            std::to_string(c.noconv_step));
    return TDCFIE_OK;
}

// Status words of the last steps of h (call after they completed)
tdcfie_status plan_check(tdcfie_t h) {
    StepPlan* p = h->plan;
    Ctl c;
    CK(cudaMemcpy(&c, p->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
    return status_of(h, c);
}

int plan_launches_per_step(tdcfie_t h) { return h->plan ? h->plan->launches_per_step : 0; }

tdcfie_status plan_step(tdcfie_t h, int64_t nsteps, void* out, void* yout) {
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
        const cudaError_t ce = capture_step(h, s);
        const cudaError_t ee = cudaStreamEndCapture(s, &p->graph);
        if (ce != cudaSuccess) {
            if (p->graph) { cudaGraphDestroy(p->graph); p->graph = nullptr; }
            return cuda_fail(h, ce, "capturing the step graph");
        }
        CK(ee);
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
    c.yout = yout;
    CK(cudaMemcpyAsync(p->ctl, &c, sizeof(Ctl), cudaMemcpyHostToDevice, s));
    long long g0[6] = {0, 0, 0, 0, 0, 0}, g1[6] = {0, 0, 0, 0, 0, 0};
    if (p->gm) CK(gmres_stats(p->gm, g0));
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
    if (p->gm) {
        CK(gmres_stats(p->gm, g1));
        h->last_launches += (g1[5] - g0[5]) * gmres_body_launches();
    }
    return status_of(h, c);
}

}  // namespace tdc
