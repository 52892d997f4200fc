// Formation of the qHP TD-CFIE blocks on the device (FP64, one-time).
//
// Projectors (Sec. II-D): P^S = Sigma (Sigma^T Sigma)^+ Sigma^T, PP^L = Lambda (Lambda^T Lambda)^+ Lambda^T,
// with L^+ = (L + 1 1^T / n)^-1 - 1 1^T / n for the (connected) graph Laplacians.
// Yukawa preconditioner and MFIE factor (Sec. III-B, III-C):
//   Z~ = (dtt PP^SH + PP^L) Zs (PP^SH + PP^L / dtt) + Zh / dtt      (PP^L Zh PP^L = Zh)
//   X~ = (dtt PP^SH + PP^L)(G/2 - M),  L1 = Z~ G^-T,  L2 = X~ G^-1
// Blocks (Sec. IV-A): with A = L1 (dtt P^LH + P^S), MM'_k = MM_k + G/2 [k = 0],
//   C_k = A S_k + alpha L2 MM'_k
//   T_k = C_k + [(1/dtt - 1) C_k - C_{k-1} / dtt] P^S + (L1 Sigma) Phi_k Sigma^T
// For the reduced-precision paths the per-lag products (everything inside the lag loop) run as
// FP32 GEMMs from FP64 operands; projector pseudo-inverses, G^-1, L1, L2 and T_0^-1 stay FP64.
// which is ZZ~_k = (dtt P^LH + P^S)[S_k P^LH + (S_k - S_{k-1}) P^S / dtt] + H_k and
// XX~_k = MM'_k (P^LH + P^S/dtt) - MM'_{k-1} P^S / dtt multiplied out in another order.
#include <utility>
#include <vector>

#include "internal.h"

namespace tdc {

// out[i][j] = beta out[i][j] + X[a[i]][j] - X[b[i]][j]        (rows of Sigma or Lambda applied on the left)
__global__ void k_g2rows(double* out, const double* X, const int* a, const int* b, int nout, int cols, double beta) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)nout * cols) return;
    const int i = (int)(t / cols), j = (int)(t % cols);
    const double v = X[(int64_t)a[i] * cols + j] - X[(int64_t)b[i] * cols + j];
    out[t] = beta == 0.0 ? v : beta * out[t] + v;
}
// out[r][i] = beta out[r][i] + X[r][a[i]] - X[r][b[i]]        (X Sigma^T / X Lambda^T)
template <typename TX>
__global__ void k_g2cols(double* out, const TX* X, const int* a, const int* b, int rows, int nout, int ldx,
                         double beta) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)rows * nout) return;
    const int r = (int)(t / nout), i = (int)(t % nout);
    const double v = (double)X[(int64_t)r * ldx + a[i]] - (double)X[(int64_t)r * ldx + b[i]];
    out[t] = beta == 0.0 ? v : beta * out[t] + v;
}
// out[i][j] = sum_e w[e] X[idx[e]][j]                          (Sigma^T X / Lambda^T X)
__global__ void k_csrrows(double* out, const double* X, const int* ptr, const int* idx, const double* w, int nout,
                          int cols) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)nout * cols) return;
    const int i = (int)(t / cols), j = (int)(t % cols);
    double s = 0.0;
    for (int e = ptr[i]; e < ptr[i + 1]; ++e) s += w[e] * X[(int64_t)idx[e] * cols + j];
    out[t] = s;
}
// out[r][i] = sum_e w[e] X[r][idx[e]]                          (X Sigma / X Lambda)
template <typename TO, typename TX>
__global__ void k_csrcols(TO* out, const TX* X, const int* ptr, const int* idx, const double* w, int rows,
                          int nout, int ldx) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)rows * nout) return;
    const int r = (int)(t / nout), i = (int)(t % nout);
    double s = 0.0;
    for (int e = ptr[i]; e < ptr[i + 1]; ++e) s += w[e] * (double)X[(int64_t)r * ldx + idx[e]];
    out[t] = (TO)s;
}
// y = a x + b y in FP32 (lag recurrence of the FP32 formation)
__global__ void k_axpby32(int64_t n, float a, const float* x, float b, float* y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = a * x[i] + b * y[i];
}
// FP64 -> FP32 copy with an optional added scaled matrix: out = (float)(X + s G)
__global__ void k_cast_add(float* out, const double* X, const double* G, double s, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)(X[i] + (G ? s * G[i] : 0.0));
}
// dense L + 1 1^T / n for a graph given by its edge list (a, b)
__global__ void k_lap_fill(double* L, int n, double val) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < (int64_t)n * n) L[t] = val;
}
__global__ void k_lap_edges(double* L, int n, const int* a, const int* b, int nedges) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nedges) return;
    atomicAdd(L + (int64_t)a[e] * n + a[e], 1.0);
    atomicAdd(L + (int64_t)b[e] * n + b[e], 1.0);
    atomicAdd(L + (int64_t)a[e] * n + b[e], -1.0);
    atomicAdd(L + (int64_t)b[e] * n + a[e], -1.0);
}
__global__ void k_axpby_f32_to_f64(int64_t n, const float* x, double* y) {   // y += x
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] += (double)x[i];
}
__global__ void k_add_scalar(double* X, int64_t n, double v) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) X[t] += v;
}
__global__ void k_add_diag_scaled(double* X, const double* G, int n, double s) {   // X += s G
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < (int64_t)n * n) X[t] += s * G[t];
}

static unsigned nb(int64_t n) { return (unsigned)((n + 255) / 256); }

struct Inc {   // sparse incidence on the device
    int *cp, *cm, *vp, *vm;                          // per edge
    int *sT_ptr, *sT_idx; double* sT_w;              // Sigma^T as CSR over triangles
    int *lT_ptr, *lT_idx; double* lT_w;              // Lambda^T as CSR over vertices
};

struct Former {
    tdcfie_t h;
    cudaStream_t s;
    int ne, nc, nv;
    Inc inc{};
    double *pinvS = nullptr, *pinvL = nullptr, *work = nullptr;
    std::vector<void*> owned;
    cudaError_t err = cudaSuccess;

    double* alloc(int64_t n) {
        void* p = nullptr;
        cudaError_t e = cudaMalloc(&p, sizeof(double) * (size_t)n);
        if (e != cudaSuccess) { err = e; return nullptr; }
        owned.push_back(p);
        return (double*)p;
    }
    void release(void* p) {
        for (auto& q : owned) if (q == p) { cudaFree(p); q = nullptr; }
    }
    ~Former() { for (void* p : owned) if (p) cudaFree(p); }

    // X (ne x cols) -> P^S X
    void PS_left(const double* X, int cols, double* out, double* tmp_nc, double* tmp_nc2) {
        k_csrrows<<<nb((int64_t)nc * cols), 256, 0, s>>>(tmp_nc, X, inc.sT_ptr, inc.sT_idx, inc.sT_w, nc, cols);
        dgemm(s, false, false, nc, cols, nc, 1.0, pinvS, nc, tmp_nc, cols, 0.0, tmp_nc2, cols);
        k_g2rows<<<nb((int64_t)ne * cols), 256, 0, s>>>(out, tmp_nc2, inc.cp, inc.cm, ne, cols, 0.0);
    }
    // X (rows x ne) -> X P^S, added as out = beta out + X P^S
    void PS_right(const double* X, int rows, double* out, double beta, double* tmp_nc, double* tmp_nc2) {
        k_csrcols<double, double><<<nb((int64_t)rows * nc), 256, 0, s>>>(tmp_nc, X, inc.sT_ptr, inc.sT_idx, inc.sT_w, rows, nc, ne);
        dgemm(s, false, false, rows, nc, nc, 1.0, tmp_nc, nc, pinvS, nc, 0.0, tmp_nc2, nc);
        k_g2cols<<<nb((int64_t)rows * ne), 256, 0, s>>>(out, (const double*)tmp_nc2, inc.cp, inc.cm, rows, ne, nc, beta);
    }
    void PL_left(const double* X, int cols, double* out, double* tmp_nv, double* tmp_nv2) {
        k_csrrows<<<nb((int64_t)nv * cols), 256, 0, s>>>(tmp_nv, X, inc.lT_ptr, inc.lT_idx, inc.lT_w, nv, cols);
        dgemm(s, false, false, nv, cols, nv, 1.0, pinvL, nv, tmp_nv, cols, 0.0, tmp_nv2, cols);
        k_g2rows<<<nb((int64_t)ne * cols), 256, 0, s>>>(out, tmp_nv2, inc.vp, inc.vm, ne, cols, 0.0);
    }
    void PL_right(const double* X, int rows, double* out, double beta, double* tmp_nv, double* tmp_nv2) {
        k_csrcols<double, double><<<nb((int64_t)rows * nv), 256, 0, s>>>(tmp_nv, X, inc.lT_ptr, inc.lT_idx, inc.lT_w, rows, nv, ne);
        dgemm(s, false, false, rows, nv, nv, 1.0, tmp_nv, nv, pinvL, nv, 0.0, tmp_nv2, nv);
        k_g2cols<<<nb((int64_t)rows * ne), 256, 0, s>>>(out, (const double*)tmp_nv2, inc.vp, inc.vm, rows, ne, nv, beta);
    }
    // (B^T B)^+ for the graph with edges (a, b) on n nodes
    bool graph_pinv(double* L, int n, const int* a, const int* b, int nedges) {
        k_lap_fill<<<nb((int64_t)n * n), 256, 0, s>>>(L, n, 1.0 / n);
        k_lap_edges<<<nb(nedges), 256, 0, s>>>(L, n, a, b, nedges);
        if (invert(s, L, n, work)) return false;
        k_add_scalar<<<nb((int64_t)n * n), 256, 0, s>>>(L, (int64_t)n * n, -1.0 / n);
        return true;
    }
};

template <class T>
static T* upload(Former& f, const std::vector<T>& v) {
    void* p = nullptr;
    if (cudaMalloc(&p, sizeof(T) * (v.size() ? v.size() : 1)) != cudaSuccess) { f.err = cudaErrorMemoryAllocation; return nullptr; }
    f.owned.push_back(p);
    cudaMemcpyAsync(p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, f.s);
    return (T*)p;
}

tdcfie_status form_operators(tdcfie_t h) {
    const Mesh& M = h->mesh;
    Former f;
    f.h = h; f.s = h->stream; f.ne = M.ne; f.nc = M.nc; f.nv = M.nv;
    const int ne = M.ne, nc = M.nc, nv = M.nv, K = h->K;
    const double dtt = h->dtt, alpha = h->alpha;
    cudaStream_t s = f.s;
    // incidence tables
    std::vector<int> cp(M.cplus), cm(M.cminus), vp(ne), vm(ne);
    for (int e = 0; e < ne; ++e) { vm[e] = M.E[2 * e]; vp[e] = M.E[2 * e + 1]; }
    std::vector<int> sptr(nc + 1), sidx(3 * nc);
    std::vector<double> sw(3 * nc);
    for (int c = 0; c <= nc; ++c) sptr[c] = 3 * c;
    for (int i = 0; i < 3 * nc; ++i) { sidx[i] = M.tedge[i]; sw[i] = M.tsign[i]; }
    std::vector<int> lptr(nv + 1, 0), lidx(2 * ne);
    std::vector<double> lw(2 * ne);
    for (int e = 0; e < ne; ++e) { lptr[vm[e] + 1]++; lptr[vp[e] + 1]++; }
    for (int v = 0; v < nv; ++v) lptr[v + 1] += lptr[v];
    {
        std::vector<int> fill(lptr.begin(), lptr.end() - 1);
        for (int e = 0; e < ne; ++e) {
            lidx[fill[vm[e]]] = e; lw[fill[vm[e]]++] = -1.0;
            lidx[fill[vp[e]]] = e; lw[fill[vp[e]]++] = +1.0;
        }
    }
    f.inc.cp = upload(f, cp); f.inc.cm = upload(f, cm); f.inc.vp = upload(f, vp); f.inc.vm = upload(f, vm);
    f.inc.sT_ptr = upload(f, sptr); f.inc.sT_idx = upload(f, sidx); f.inc.sT_w = upload(f, sw);
    f.inc.lT_ptr = upload(f, lptr); f.inc.lT_idx = upload(f, lidx); f.inc.lT_w = upload(f, lw);
    const int nmax = std::max(ne, std::max(nc, nv));
    f.work = f.alloc(2 * (int64_t)nmax + 2);
    // pseudo-inverses of the graph Laplacians
    if (!h->PinvS && cudaMalloc(&h->PinvS, sizeof(double) * (size_t)nc * nc) != cudaSuccess)
        return fail(h, TDCFIE_E_OOM, "PinvS");
    f.pinvS = h->PinvS;
    f.pinvL = f.alloc((int64_t)nv * nv);
    if (f.err != cudaSuccess) return cuda_fail(h, f.err, "formation allocation");
    if (!f.graph_pinv(f.pinvS, nc, f.inc.cp, f.inc.cm, ne)) return fail(h, TDCFIE_E_MESH, "dual graph Laplacian singular");
    if (!f.graph_pinv(f.pinvL, nv, f.inc.vp, f.inc.vm, ne)) return fail(h, TDCFIE_E_MESH, "vertex graph Laplacian singular");
    const int64_t NN = (int64_t)ne * ne;
    double* tnc = f.alloc((int64_t)ne * std::max(nc, nv));
    double* tnc2 = f.alloc((int64_t)ne * std::max(nc, nv));
    double* Y = f.alloc(NN);
    double* Z = f.alloc(NN);
    if (f.err != cudaSuccess) return cuda_fail(h, f.err, "formation allocation");
    // Zh = Lambda Psi Lambda^T
    double* LPsi = f.alloc((int64_t)ne * nv);
    if (!h->Zh && cudaMalloc(&h->Zh, sizeof(double) * NN) != cudaSuccess) return fail(h, TDCFIE_E_OOM, "Zh");
    k_g2rows<<<nb((int64_t)ne * nv), 256, 0, s>>>(LPsi, h->Psi, f.inc.vp, f.inc.vm, ne, nv, 0.0);
    k_g2cols<double><<<nb(NN), 256, 0, s>>>(h->Zh, (const double*)LPsi, f.inc.vp, f.inc.vm, ne, ne, nv, 0.0);
    f.release(LPsi);
    // Z~ = dtt Y + (1 - dtt) PP^L Y + Zh/dtt,   Y = Zs + (1/dtt - 1) Zs PP^L
    cudaMemcpyAsync(Y, h->Zs, sizeof(double) * NN, cudaMemcpyDeviceToDevice, s);
    f.PL_right(h->Zs, ne, Z, 0.0, tnc, tnc2);
    axpby(s, NN, 1.0 / dtt - 1.0, Z, 1.0, Y);
    f.PL_left(Y, ne, Z, tnc, tnc2);
    double* Zt = f.alloc(NN);
    cudaMemcpyAsync(Zt, Y, sizeof(double) * NN, cudaMemcpyDeviceToDevice, s);
    axpby(s, NN, 1.0 - dtt, Z, dtt, Zt);
    axpby(s, NN, 1.0 / dtt, h->Zh, 1.0, Zt);
    // X~ = dtt X0 + (1 - dtt) PP^L X0,  X0 = G/2 - M
    axpby(s, NN, 0.5, h->G, 0.0, Y);
    axpby(s, NN, -1.0, h->Mst, 1.0, Y);
    f.PL_left(Y, ne, Z, tnc, tnc2);
    axpby(s, NN, 1.0 - dtt, Z, dtt, Y);   // Y = X~
    // G^-1
    double* Ginv = f.alloc(NN);
    if (f.err != cudaSuccess) return cuda_fail(h, f.err, "formation allocation");
    cudaMemcpyAsync(Ginv, h->G, sizeof(double) * NN, cudaMemcpyDeviceToDevice, s);
    if (invert(s, Ginv, ne, f.work)) return fail(h, TDCFIE_E_MESH, "Gram matrix singular");
    if (!h->L1) cudaMalloc(&h->L1, sizeof(double) * NN);
    if (!h->L2) cudaMalloc(&h->L2, sizeof(double) * NN);
    if (!h->A) cudaMalloc(&h->A, sizeof(double) * NN);
    if (!h->L1 || !h->L2 || !h->A) return fail(h, TDCFIE_E_OOM, "L1/L2/A");
    dgemm(s, false, true, ne, ne, ne, 1.0, Zt, ne, Ginv, ne, 0.0, h->L1, ne);   // L1 = Z~ G^-T
    dgemm(s, false, false, ne, ne, ne, 1.0, Y, ne, Ginv, ne, 0.0, h->L2, ne);    // L2 = X~ G^-1
    f.release(Zt);
    f.release(Ginv);
    // A = dtt L1 + (1 - dtt) L1 P^S
    f.PS_right(h->L1, ne, Z, 0.0, tnc, tnc2);   // Z = L1 P^S
    cudaMemcpyAsync(h->A, h->L1, sizeof(double) * NN, cudaMemcpyDeviceToDevice, s);
    axpby(s, NN, 1.0 - dtt, Z, dtt, h->A);
    // L1 Sigma (ne x nc)
    double* L1S = f.alloc((int64_t)ne * nc);
    double* Ek = f.alloc((int64_t)ne * nc);
    double* Cprev = f.alloc(NN);
    double* Ck = f.alloc(NN);
    if (f.err != cudaSuccess) return cuda_fail(h, f.err, "formation allocation");
    k_csrcols<double, double><<<nb((int64_t)ne * nc), 256, 0, s>>>(L1S, h->L1, f.inc.sT_ptr, f.inc.sT_idx, f.inc.sT_w, ne, nc, ne);
    if (!h->T && cudaMalloc(&h->T, sizeof(double) * NN * K) != cudaSuccess) return fail(h, TDCFIE_E_OOM, "T_k");
    const bool f32 = h->opts.precision != TDCFIE_FP64;
    if (!f32) {
        cudaMemsetAsync(Cprev, 0, sizeof(double) * NN, s);
        for (int k = 0; k < K; ++k) {
            double* MMk = h->MM + (int64_t)k * NN;
            if (k == 0) k_add_diag_scaled<<<nb(NN), 256, 0, s>>>(MMk, h->G, ne, 0.5);   // MM'_0 = MM_0 + G/2
            dgemm(s, false, false, ne, ne, ne, 1.0, h->A, ne, h->S + (int64_t)k * NN, ne, 0.0, Ck, ne);
            dgemm(s, false, false, ne, ne, ne, alpha, h->L2, ne, MMk, ne, 1.0, Ck, ne);
            if (k == 0) k_add_diag_scaled<<<nb(NN), 256, 0, s>>>(MMk, h->G, ne, -0.5);  // restore MM_0
            // D_k = (1/dtt - 1) C_k - C_{k-1}/dtt  (into Cprev, which is free afterwards)
            axpby(s, NN, 1.0 / dtt - 1.0, Ck, -1.0 / dtt, Cprev);
            // E_k = (D_k Sigma) (Sigma^T Sigma)^+ + (L1 Sigma) Phi_k
            k_csrcols<double, double><<<nb((int64_t)ne * nc), 256, 0, s>>>(tnc, Cprev, f.inc.sT_ptr, f.inc.sT_idx,
                                                                          f.inc.sT_w, ne, nc, ne);
            dgemm(s, false, false, ne, nc, nc, 1.0, tnc, nc, f.pinvS, nc, 0.0, Ek, nc);
            dgemm(s, false, false, ne, nc, nc, 1.0, L1S, nc, h->Phi + (int64_t)k * nc * nc, nc, 1.0, Ek, nc);
            double* Tk = h->T + (int64_t)k * NN;
            cudaMemcpyAsync(Tk, Ck, sizeof(double) * NN, cudaMemcpyDeviceToDevice, s);
            k_g2cols<double><<<nb(NN), 256, 0, s>>>(Tk, (const double*)Ek, f.inc.cp, f.inc.cm, ne, ne, nc, 1.0);
            std::swap(Cprev, Ck);
        }
    } else {
        // FP32 products: operands cast once (A, L2, L1 Sigma, pinv) or per lag (S_k, MM'_k, Phi_k)
        float* fb = nullptr;
        const int64_t need = 6 * NN + 3 * (int64_t)ne * nc + 2 * (int64_t)nc * nc;
        if (cudaMalloc(&fb, sizeof(float) * need) != cudaSuccess) return fail(h, TDCFIE_E_OOM, "FP32 formation");
        f.owned.push_back(fb);
        float *Af = fb, *L2f = Af + NN, *Sf = L2f + NN, *Mf = Sf + NN, *Cf = Mf + NN, *Cpf = Cf + NN;
        float *L1Sf = Cpf + NN, *Df = L1Sf + (int64_t)ne * nc, *Ef = Df + (int64_t)ne * nc;
        float *Pf = Ef + (int64_t)ne * nc, *Phf = Pf + (int64_t)nc * nc;
        k_cast_add<<<nb(NN), 256, 0, s>>>(Af, h->A, nullptr, 0.0, NN);
        k_cast_add<<<nb(NN), 256, 0, s>>>(L2f, h->L2, nullptr, 0.0, NN);
        k_cast_add<<<nb((int64_t)ne * nc), 256, 0, s>>>(L1Sf, L1S, nullptr, 0.0, (int64_t)ne * nc);
        k_cast_add<<<nb((int64_t)nc * nc), 256, 0, s>>>(Pf, f.pinvS, nullptr, 0.0, (int64_t)nc * nc);
        cudaMemsetAsync(Cpf, 0, sizeof(float) * NN, s);
        for (int k = 0; k < K; ++k) {
            k_cast_add<<<nb(NN), 256, 0, s>>>(Sf, h->S + (int64_t)k * NN, nullptr, 0.0, NN);
            k_cast_add<<<nb(NN), 256, 0, s>>>(Mf, h->MM + (int64_t)k * NN, k == 0 ? h->G : nullptr, 0.5, NN);
            k_cast_add<<<nb((int64_t)nc * nc), 256, 0, s>>>(Phf, h->Phi + (int64_t)k * nc * nc, nullptr, 0.0,
                                                            (int64_t)nc * nc);
            sgemm(s, false, false, ne, ne, ne, 1.f, Af, ne, Sf, ne, 0.f, Cf, ne);
            sgemm(s, false, false, ne, ne, ne, (float)alpha, L2f, ne, Mf, ne, 1.f, Cf, ne);
            k_axpby32<<<nb(NN), 256, 0, s>>>(NN, (float)(1.0 / dtt - 1.0), Cf, (float)(-1.0 / dtt), Cpf);
            k_csrcols<float, float><<<nb((int64_t)ne * nc), 256, 0, s>>>(Df, Cpf, f.inc.sT_ptr, f.inc.sT_idx,
                                                                        f.inc.sT_w, ne, nc, ne);
            sgemm(s, false, false, ne, nc, nc, 1.f, Df, nc, Pf, nc, 0.f, Ef, nc);
            sgemm(s, false, false, ne, nc, nc, 1.f, L1Sf, nc, Phf, nc, 1.f, Ef, nc);
            double* Tk = h->T + (int64_t)k * NN;
            k_g2cols<float><<<nb(NN), 256, 0, s>>>(Tk, Ef, f.inc.cp, f.inc.cm, ne, ne, nc, 0.0);
            k_axpby_f32_to_f64<<<nb(NN), 256, 0, s>>>(NN, Cf, Tk);
            std::swap(Cpf, Cf);
        }
    }
    // T_0^-1
    if (!h->T0inv && cudaMalloc(&h->T0inv, sizeof(double) * NN) != cudaSuccess) return fail(h, TDCFIE_E_OOM, "T0inv");
    cudaMemcpyAsync(h->T0inv, h->T, sizeof(double) * NN, cudaMemcpyDeviceToDevice, s);
    if (invert(s, h->T0inv, ne, f.work)) return fail(h, TDCFIE_E_STATE, "T_0 is singular");
    // dense P^S (kept for inspection)
    if (!h->PS && cudaMalloc(&h->PS, sizeof(double) * NN) != cudaSuccess) return fail(h, TDCFIE_E_OOM, "PS");
    fill_identity(s, Y, ne, 1.0);
    f.PS_left(Y, ne, h->PS, tnc, tnc2);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(h, e, "formation");
    return TDCFIE_OK;
}

}  // namespace tdc
