// Factored history form of the MOT step (Sec. IV-A, Eq. dis_TD_CFIE, and Sec. IV-B), FP64 and FP32.
//
// The dense blocks T_k are products of the retarded matrices with dense static factors:
//   sum_{k>=1} T_k y_{n-k} = A es + L1 Sigma eh + alpha L2 mm,    A = L1 (dtt P^LH + P^S),
//   es = sum_{k>=0} S_k x_{n-k},  mm = sum_{k>=0} MM'_k x_{n-k},  eh = sum_{k>=1} Phi_k q_{n-k},
// with x_{n-k} = j_{n-k} (k >= 1) the physical currents of Eq. post_processing, x_n = c_n =
// -P^S y_{n-1} / dtt (the part of j_n that is known before y_n), MM'_k = MM_k + G/2 [k = 0], and
// q_i = Sigma^T y_i the charges (H_k = Sigma Phi_k Sigma^T).  S_k, MM'_k and Phi_k are shell-sparse:
// an entry is nonzero only for the few lags k whose time-basis support meets the distances of the
// two basis functions, so that sum_k nnz is a few N^2 for every K, against K N^2 for the T_k.
//
// Per step n (one CUDA graph):
//   rhs       e_n, h_n (the plane-wave tests of the dense path)
//   shells    z = [e_n + es ; h_n - mm ; eh]   (one warp per row of [S ; -MM' ; Phi], all lags)
//   solve     y_n = W z,  W = T_0^-1 [-A | alpha L2 | -L1 Sigma]   (formed once in FP64)
//   charges   q_n = Sigma^T y_n
//   pinv      v_n = (Sigma^T Sigma)^+ q_n,     so that P^S y_n = Sigma v_n
//   post      j_n = y_n + Sigma ((1/dtt - 1) v_n - v_{n-1} / dtt),  c_{n+1} = -Sigma v_n / dtt
// Rings (HBM, right-hand-side-major as in the dense path): x ring of K slots (slot i mod K holds
// j_i, and c_n in slot n mod K while step n runs), q ring of K slots, y and v of 2 slots.
//
// Shell storage: one CSR over the 2 ne + nc rows, each row's entries ordered by (lag, column),
// packed index (k << 24) | column, rows padded to a multiple of 4 entries (zero values) so that
// every row starts on a 16-byte boundary of both arrays.  K <= 256 and ne < 2^24.
#include <algorithm>
#include <vector>

#include "internal.h"
#include "plan.h"
#include "simt.h"

namespace tdc {

struct FactPlan {
    int K = 0, nrows = 0, ldz = 0;
    int64_t nnz = 0;            // stored entries (with the row padding)
    int64_t nnz_true = 0;       // nonzeros of S_k, MM'_k, Phi_k
    int64_t* rowptr = nullptr;  // nrows + 1
    uint32_t* idx = nullptr;    // nnz
    void* val = nullptr;        // nnz (path precision)
    void* W = nullptr;          // ne x ldz (path precision)
    void* xring = nullptr;      // K x R x ne
    void* qring = nullptr;      // K x R x nc
    void* qcur = nullptr;       // R x nc
    void* y2 = nullptr;         // 2 x R x ne
    void* v2 = nullptr;         // 2 x R x nc
    void* z = nullptr;          // R x ldz
};

// ---------------------------------------------------------------- construction
// Row r of the stacked operator: S (r < ne), -MM' (ne <= r < 2 ne), Phi (r >= 2 ne, lags >= 1).
struct ShellSrc {
    const double* S; const double* MM; const double* G; const double* Phi;
    int ne, nc, K;
    __device__ int ncols(int r) const { return r < 2 * ne ? ne : nc; }
    __device__ int k0(int r) const { return r < 2 * ne ? 0 : 1; }
    __device__ double value(int r, int k, int col) const {
        if (r < ne) return S[((int64_t)k * ne + r) * ne + col];
        if (r < 2 * ne) {
            const int i = r - ne;
            double v = MM[((int64_t)k * ne + i) * ne + col];
            if (k == 0) v += 0.5 * G[(int64_t)i * ne + col];
            return -v;
        }
        const int c = r - 2 * ne;
        return Phi[((int64_t)k * nc + c) * nc + col];
    }
};

__global__ void k_shell_count(ShellSrc src, int nrows, int64_t* cnt) {
    const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= nrows) return;
    const int nc = src.ncols(r);
    int64_t c = 0;
    for (int k = src.k0(r); k < src.K; ++k)
        for (int col = lane; col < nc; col += 32) c += src.value(r, k, col) != 0.0;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) cnt[r] = c;
}

template <typename T>
__global__ void k_shell_fill(ShellSrc src, int nrows, const int64_t* __restrict__ rowptr, uint32_t* __restrict__ idx,
                             T* __restrict__ val) {
    const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= nrows) return;
    const int nc = src.ncols(r);
    int64_t pos = rowptr[r];
    for (int k = src.k0(r); k < src.K; ++k)
        for (int c0 = 0; c0 < nc; c0 += 32) {
            const int col = c0 + lane;
            const double v = col < nc ? src.value(r, k, col) : 0.0;
            const unsigned m = __ballot_sync(0xffffffffu, v != 0.0);
            if (v != 0.0) {
                const int64_t at = pos + __popc(m & ((1u << lane) - 1u));
                idx[at] = ((uint32_t)k << 24) | (uint32_t)col;
                val[at] = (T)v;
            }
            pos += __popc(m);
        }
    // padding up to the next multiple of 4: zero values on lag 0, column 0
    for (int64_t at = pos + lane; at < rowptr[r + 1]; at += 32) {
        idx[at] = 0u;
        val[at] = (T)0;
    }
}

// B = [-A | alpha L2 | -L1 Sigma | 0] (ne x ldz), (L1 Sigma)[i][c] = sum_j tsign[c][j] L1[i][tedge[c][j]]
__global__ void k_fact_bcat(DevMesh m, int ldz, const double* __restrict__ A, const double* __restrict__ L2,
                            const double* __restrict__ L1, double alpha, double* __restrict__ B) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int ne = m.ne, nc = m.nc;
    if (t >= (int64_t)ne * ldz) return;
    const int i = (int)(t / ldz), col = (int)(t % ldz);
    double v = 0.0;
    if (col < ne) v = -A[(int64_t)i * ne + col];
    else if (col < 2 * ne) v = alpha * L2[(int64_t)i * ne + col - ne];
    else if (col < 2 * ne + nc) {
        const int c = col - 2 * ne;
        double s = 0.0;
        for (int j = 0; j < 3; ++j) s += m.tsign[3 * c + j] * L1[(int64_t)i * ne + m.tedge[3 * c + j]];
        v = -s;
    }
    B[t] = v;
}

// ---------------------------------------------------------------- step kernels
// z[r][row] = base[r][i] + sum over the row's entries of val * x_{n-k}[r][col]
template <typename T>
struct ShellDot;

template <>
struct ShellDot<double> {
    template <int RMAX>
    __device__ static void run(const uint32_t* __restrict__ idx, const double* __restrict__ val, int64_t b, int64_t e,
                               const double* __restrict__ ring, int64_t slot_stride, int ld, int nb, int K, int R,
                               int tid, int step, double* acc) {
        double s[RMAX];
#pragma unroll
        for (int r = 0; r < RMAX; ++r) s[r] = 0.0;
        for (int64_t p = b + 4 * tid; p < e; p += step) {
            const uint4 ix = *reinterpret_cast<const uint4*>(idx + p);
            const double2 v01 = *reinterpret_cast<const double2*>(val + p);
            const double2 v23 = *reinterpret_cast<const double2*>(val + p + 2);
            const uint32_t ii[4] = {ix.x, ix.y, ix.z, ix.w};
            const double vv[4] = {v01.x, v01.y, v23.x, v23.y};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                int slot = nb - (int)(ii[u] >> 24);
                if (slot < 0) slot += K;
                const double* x = ring + slot * slot_stride + (ii[u] & 0xFFFFFFu);
#pragma unroll
                for (int r = 0; r < RMAX; ++r)
                    if (r < R) s[r] = fma(vv[u], x[(int64_t)r * ld], s[r]);
            }
        }
#pragma unroll
        for (int r = 0; r < RMAX; ++r) {
            double v = s[r];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            acc[r] = v;
        }
    }
};

template <>
struct ShellDot<float> {
    // error-free products and sums as in the dense FP32 row sums (RowDot<float>)
    template <int RMAX>
    __device__ static void run(const uint32_t* __restrict__ idx, const float* __restrict__ val, int64_t b, int64_t e,
                               const float* __restrict__ ring, int64_t slot_stride, int ld, int nb, int K, int R,
                               int tid, int step, double* acc) {
        float hi[RMAX], lo[RMAX];
#pragma unroll
        for (int r = 0; r < RMAX; ++r) hi[r] = lo[r] = 0.f;
        for (int64_t p = b + 4 * tid; p < e; p += step) {
            const uint4 ix = *reinterpret_cast<const uint4*>(idx + p);
            const float4 v4 = *reinterpret_cast<const float4*>(val + p);
            const uint32_t ii[4] = {ix.x, ix.y, ix.z, ix.w};
            const float vv[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                int slot = nb - (int)(ii[u] >> 24);
                if (slot < 0) slot += K;
                const float* x = ring + slot * slot_stride + (ii[u] & 0xFFFFFFu);
#pragma unroll
                for (int r = 0; r < RMAX; ++r)
                    if (r < R) ff_add(hi[r], lo[r], vv[u], x[(int64_t)r * ld]);
            }
        }
#pragma unroll
        for (int r = 0; r < RMAX; ++r) {
            double v = (double)hi[r] + (double)lo[r];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            acc[r] = v;
        }
    }
};

// WPR warps per row (a row holds every lag of one basis function: thousands of entries), partial
// sums combined through shared memory in a fixed order
constexpr int WPR = 4;

template <typename T, int RMAX>
__global__ void __launch_bounds__(256) k_shells(int ne, int nc, int K, int R, int ldz, const Ctl* ctl,
                                                const int64_t* __restrict__ rowptr, const uint32_t* __restrict__ idx,
                                                const T* __restrict__ val, const T* __restrict__ xring,
                                                const T* __restrict__ qring, const T* __restrict__ E,
                                                const T* __restrict__ Hv, T* __restrict__ z) {
    __shared__ double part[256 / 32][RMAX];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = blockIdx.x * (256 / 32 / WPR) + warp / WPR;
    const int w = warp % WPR;
    const bool live = row < 2 * ne + nc;
    double acc[RMAX];
    if (live) {
        const int nb = (int)(ctl->n % K);
        const bool charge = row >= 2 * ne;
        const T* ring = charge ? qring : xring;
        const int ld = charge ? nc : ne;
        ShellDot<T>::template run<RMAX>(idx, val, rowptr[row], rowptr[row + 1], ring, (int64_t)R * ld, ld, nb, K, R,
                                        w * 32 + lane, 128 * WPR, acc);
        if (lane == 0) {
#pragma unroll
            for (int r = 0; r < RMAX; ++r) part[warp][r] = acc[r];
        }
    }
    __syncthreads();
    if (live && w == 0 && lane < R) {
        double v = 0.0;
        for (int q = 0; q < WPR; ++q) v += part[warp + q][lane];
        double base = 0.0;
        if (row < ne) base = (double)E[(int64_t)lane * ne + row];
        else if (row < 2 * ne) base = (double)Hv[(int64_t)lane * ne + row - ne];
        z[(int64_t)lane * ldz + row] = (T)(base + v);
    }
}

// q_n = Sigma^T y_n into the charge ring and qcur
template <typename T>
__global__ void k_fact_charges(DevMesh m, int R, int K, const Ctl* ctl, const T* __restrict__ y2, T* __restrict__ qring,
                               T* __restrict__ qcur) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m.nc * R) return;
    const int r = t / m.nc, c = t % m.nc;
    const int64_t n = ctl->n;
    const T* y = y2 + (n & 1) * (int64_t)R * m.ne + (int64_t)r * m.ne;
    double s = 0.0;
    for (int j = 0; j < 3; ++j) s = fma(m.tsign[3 * c + j], (double)y[m.tedge[3 * c + j]], s);
    const T q = (T)s;
    qring[((n % K) * R + r) * (int64_t)m.nc + c] = q;
    qcur[(int64_t)r * m.nc + c] = q;
}

// j_n = y_n + Sigma((1/dtt - 1) v_n - v_{n-1}/dtt) -> x ring slot n, outputs; c_{n+1} -> slot n+1
template <typename T>
__global__ void k_fact_post(DevMesh m, int R, int K, Ctl* ctl, const T* __restrict__ y2, const T* __restrict__ v2,
                            T* __restrict__ xring, double dtt) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m.ne * R) return;
    const int r = t / m.ne, e = t % m.ne;
    const int64_t n = ctl->n;
    const T* y = y2 + (n & 1) * (int64_t)R * m.ne + (int64_t)r * m.ne;
    const T* vn = v2 + (n & 1) * (int64_t)R * m.nc + (int64_t)r * m.nc;
    const T* vp = v2 + ((n - 1) & 1) * (int64_t)R * m.nc + (int64_t)r * m.nc;
    const int cp = m.cplus_[e], cm = m.cminus_[e];
    const double sv = (double)vn[cp] - (double)vn[cm];          // (Sigma v_n)[e]
    const double sp = (double)vp[cp] - (double)vp[cm];          // (Sigma v_{n-1})[e]
    const double jn = (double)y[e] + fma(1.0 / dtt - 1.0, sv, -sp / dtt);
    const T jv = (T)jn;
    xring[((n % K) * R + r) * (int64_t)m.ne + e] = jv;
    xring[(((n + 1) % K) * R + r) * (int64_t)m.ne + e] = (T)(-sv / dtt);
    if (!isfinite(jn) && atomicCAS(&ctl->status, 0, (int)TDCFIE_E_NONFINITE) == 0) ctl->bad_step = n;
    if (ctl->out) reinterpret_cast<T*>(ctl->out)[((n - ctl->n0) * R + r) * (int64_t)m.ne + e] = jv;
    if (ctl->yout) reinterpret_cast<T*>(ctl->yout)[((n - ctl->n0) * R + r) * (int64_t)m.ne + e] = y[e];
}

// y = M x for one matrix, one warp per row, result into slot n mod 2 of a two-slot buffer
template <typename T, int RMAX>
__global__ void k_fact_apply(const T* __restrict__ Mtx, int nrow, int ncol, int R, const T* __restrict__ x,
                             T* __restrict__ y2, const Ctl* ctl) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (warp >= nrow) return;
    double acc[RMAX];
    warp_rows<T, RMAX>(Mtx + (int64_t)warp * ncol, ncol, x, R, ncol, acc);
    T* dst = y2 + (ctl->n & 1) * (int64_t)R * nrow;
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int r = 0; r < RMAX; ++r)
            if (r < R) dst[(int64_t)r * nrow + warp] = (T)acc[r];
    }
}

__global__ void k_fact_advance(Ctl* ctl) { ctl->n += 1; }

// ---------------------------------------------------------------- host side
#define FK(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) return cuda_fail(h, e_, #x); } while (0)

void destroy_fact(FactPlan* f) {
    if (!f) return;
    void* bufs[] = {f->rowptr, f->idx, f->val, f->W, f->xring, f->qring, f->qcur, f->y2, f->v2, f->z};
    for (void* b : bufs) if (b) cudaFree(b);
    delete f;
}

tdcfie_status build_fact(tdcfie_t h, StepPlan* p) {
    cudaStream_t s = h->stream;
    const int ne = p->ne, nc = p->nc, K = p->K, R = p->R;
    const size_t es = p->esz;
    if (K > 256) return fail(h, TDCFIE_E_UNSUPPORTED, "the factored form packs the lag in 8 bits (K <= 256)");
    if (ne >= (1 << 24)) return fail(h, TDCFIE_E_UNSUPPORTED, "the factored form packs the column in 24 bits");
    if (!h->S || !h->MM || !h->Phi || !h->G || !h->T0inv || !h->A || !h->L2 || !h->L1 || !h->PinvS)
        return fail(h, TDCFIE_E_STATE, "the factored form needs the FP64 assembly");
    FactPlan* f = new FactPlan();
    p->fact = f;
    f->K = K;
    f->nrows = 2 * ne + nc;
    f->ldz = (f->nrows + 3) / 4 * 4;
    // shell CSR: count, scan on the host, fill
    ShellSrc src{h->S, h->MM, h->G, h->Phi, ne, nc, K};
    int64_t* cnt = nullptr;
    FK(cudaMalloc(&cnt, sizeof(int64_t) * f->nrows));
    const int wpb = 8;
    const unsigned gr = (unsigned)((f->nrows + wpb - 1) / wpb);
    k_shell_count<<<gr, 32 * wpb, 0, s>>>(src, f->nrows, cnt);
    FK(cudaGetLastError());
    std::vector<int64_t> hc(f->nrows), ptr(f->nrows + 1, 0);
    FK(cudaMemcpyAsync(hc.data(), cnt, sizeof(int64_t) * f->nrows, cudaMemcpyDeviceToHost, s));
    FK(cudaStreamSynchronize(s));
    cudaFree(cnt);
    for (int r = 0; r < f->nrows; ++r) {
        f->nnz_true += hc[r];
        ptr[r + 1] = ptr[r] + (hc[r] + 3) / 4 * 4;
    }
    f->nnz = ptr[f->nrows];
    FK(cudaMalloc(&f->rowptr, sizeof(int64_t) * (f->nrows + 1)));
    FK(cudaMalloc(&f->idx, sizeof(uint32_t) * std::max<int64_t>(f->nnz, 4)));
    FK(cudaMalloc(&f->val, es * std::max<int64_t>(f->nnz, 4)));
    FK(cudaMemcpyAsync(f->rowptr, ptr.data(), sizeof(int64_t) * (f->nrows + 1), cudaMemcpyHostToDevice, s));
    if (p->prec == TDCFIE_FP64) k_shell_fill<double><<<gr, 32 * wpb, 0, s>>>(src, f->nrows, f->rowptr, f->idx, (double*)f->val);
    else k_shell_fill<float><<<gr, 32 * wpb, 0, s>>>(src, f->nrows, f->rowptr, f->idx, (float*)f->val);
    FK(cudaGetLastError());
    // W = T_0^-1 [-A | alpha L2 | -L1 Sigma], formed in FP64 and stored in the path precision
    const int64_t nW = (int64_t)ne * f->ldz;
    double *B = nullptr, *W64 = nullptr;
    FK(cudaMalloc(&B, 8 * nW));
    FK(cudaMalloc(&W64, 8 * nW));
    k_fact_bcat<<<(unsigned)((nW + 255) / 256), 256, 0, s>>>(h->dm, f->ldz, h->A, h->L2, h->L1, h->alpha, B);
    FK(cudaGetLastError());
    dgemm(s, false, false, ne, f->ldz, ne, 1.0, h->T0inv, ne, B, f->ldz, 0.0, W64, f->ldz);
    FK(cudaMalloc(&f->W, es * nW));
    if (p->prec == TDCFIE_FP64) FK(cudaMemcpyAsync(f->W, W64, 8 * nW, cudaMemcpyDeviceToDevice, s));
    else cast_f64_f32(s, W64, (float*)f->W, nW);
    FK(cudaMalloc(&p->pinv, es * (int64_t)nc * nc));
    if (p->prec == TDCFIE_FP64) FK(cudaMemcpyAsync(p->pinv, h->PinvS, 8 * (int64_t)nc * nc, cudaMemcpyDeviceToDevice, s));
    else cast_f64_f32(s, h->PinvS, (float*)p->pinv, (int64_t)nc * nc);
    FK(cudaStreamSynchronize(s));
    cudaFree(B);
    cudaFree(W64);
    // march state
    FK(cudaMalloc(&f->xring, es * K * R * ne));
    FK(cudaMalloc(&f->qring, es * K * R * nc));
    FK(cudaMalloc(&f->qcur, es * R * nc));
    FK(cudaMalloc(&f->y2, es * 2 * R * ne));
    FK(cudaMalloc(&f->v2, es * 2 * R * nc));
    FK(cudaMalloc(&f->z, es * R * f->ldz));
    FK(cudaMemsetAsync(f->z, 0, es * R * f->ldz, s));   // the padding columns stay zero
    h->hist_bytes = (double)f->nnz * (4.0 + es);
    return TDCFIE_OK;
}

tdcfie_status reset_fact(tdcfie_t h, StepPlan* p) {
    FactPlan* f = p->fact;
    cudaStream_t s = h->stream;
    const size_t es = p->esz;
    FK(cudaMemsetAsync(f->xring, 0, es * f->K * p->R * p->ne, s));
    FK(cudaMemsetAsync(f->qring, 0, es * f->K * p->R * p->nc, s));
    FK(cudaMemsetAsync(f->y2, 0, es * 2 * p->R * p->ne, s));
    FK(cudaMemsetAsync(f->v2, 0, es * 2 * p->R * p->nc, s));
    return TDCFIE_OK;
}

double fact_step_bytes(const StepPlan* p) {
    const FactPlan* f = p->fact;
    return (double)f->nnz * (4.0 + p->esz) + (double)p->ne * f->ldz * p->esz + (double)p->nc * p->nc * p->esz;
}

int64_t fact_nnz(const StepPlan* p, bool stored) { return stored ? p->fact->nnz : p->fact->nnz_true; }

template <typename T, int RMAX>
static void launch_fact_r(tdcfie_t h, StepPlan& p, cudaStream_t s) {
    FactPlan& f = *p.fact;
    const tdc::DevMesh& m = h->dm;
    const int ne = p.ne, nc = p.nc, R = p.R, tb = 256, wpb = 8;
    launch_rhs<T>(h, p, s);
    cudaEventRecordWithFlags(p.evA, s, cudaEventRecordExternal);
    k_shells<T, RMAX><<<(f.nrows + wpb / WPR - 1) / (wpb / WPR), 32 * wpb, 0, s>>>(ne, nc, f.K, R, f.ldz, p.ctl, f.rowptr, f.idx,
                                                                      (const T*)f.val, (const T*)f.xring,
                                                                      (const T*)f.qring, (const T*)p.E,
                                                                      (const T*)p.Hv, (T*)f.z);
    cudaEventRecordWithFlags(p.evB, s, cudaEventRecordExternal);
    k_fact_apply<T, RMAX><<<(ne + wpb - 1) / wpb, 32 * wpb, 0, s>>>((const T*)f.W, ne, f.ldz, R, (const T*)f.z,
                                                                     (T*)f.y2, p.ctl);
    k_fact_charges<T><<<(nc * R + tb - 1) / tb, tb, 0, s>>>(m, R, f.K, p.ctl, (const T*)f.y2, (T*)f.qring, (T*)f.qcur);
    k_fact_apply<T, RMAX><<<(nc + wpb - 1) / wpb, 32 * wpb, 0, s>>>((const T*)p.pinv, nc, nc, R, (const T*)f.qcur,
                                                                     (T*)f.v2, p.ctl);
    k_fact_post<T><<<(ne * R + tb - 1) / tb, tb, 0, s>>>(m, R, f.K, p.ctl, (const T*)f.y2, (const T*)f.v2,
                                                         (T*)f.xring, h->dtt);
    k_fact_advance<<<1, 1, 0, s>>>(p.ctl);
    p.launches_per_step = 7;
}

template <typename T>
cudaError_t launch_step_fact(tdcfie_t h, StepPlan& p, cudaStream_t s) {
    if (p.R == 1) launch_fact_r<T, 1>(h, p, s);
    else if (p.R <= 4) launch_fact_r<T, 4>(h, p, s);
    else launch_fact_r<T, 8>(h, p, s);
    return cudaGetLastError();
}

template cudaError_t launch_step_fact<double>(tdcfie_t, StepPlan&, cudaStream_t);
template cudaError_t launch_step_fact<float>(tdcfie_t, StepPlan&, cudaStream_t);

}  // namespace tdc
