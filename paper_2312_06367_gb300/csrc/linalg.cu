// Dense FP64 helpers for the one-time assembly: row-major DGEMM (cuBLAS, plain library GEMM),
// in-place Gauss-Jordan inversion with partial pivoting, incidence gathers, precision casts.
#include <cublas_v2.h>
#include <cuda_bf16.h>

#include <map>

#include "internal.h"

namespace tdc {

static cublasHandle_t blas_for(cudaStream_t s) {
    static std::map<cudaStream_t, cublasHandle_t> handles;
    auto it = handles.find(s);
    if (it != handles.end()) return it->second;
    cublasHandle_t h;
    cublasCreate(&h);
    cublasSetStream(h, s);
    cublasSetMathMode(h, CUBLAS_PEDANTIC_MATH);
    handles[s] = h;
    return h;
}

// Row-major C (m x n) = alpha op(A) op(B) + beta C  <=>  column-major C^T = op(B)^T op(A)^T.
void dgemm(cudaStream_t s, bool ta, bool tb, int m, int n, int k, double alpha, const double* A, int lda,
           const double* B, int ldb, double beta, double* C, int ldc) {
    cublasDgemm(blas_for(s), tb ? CUBLAS_OP_T : CUBLAS_OP_N, ta ? CUBLAS_OP_T : CUBLAS_OP_N, n, m, k, &alpha, B, ldb,
                A, lda, &beta, C, ldc);
}

// Row-major FP32 C (m x n) = alpha op(A) op(B) + beta C (cuBLAS SGEMM, pedantic FP32: no TF32).
void sgemm(cudaStream_t s, bool ta, bool tb, int m, int n, int k, float alpha, const float* A, int lda,
           const float* B, int ldb, float beta, float* C, int ldc) {
    cublasSgemm(blas_for(s), tb ? CUBLAS_OP_T : CUBLAS_OP_N, ta ? CUBLAS_OP_T : CUBLAS_OP_N, n, m, k, &alpha, B, ldb,
                A, lda, &beta, C, ldc);
}

// ---------------------------------------------------------------- Gauss-Jordan inverse
// One block: find the pivot of column p among rows >= p, swap rows, scale the pivot row and save
// the old column p (multipliers) in f.
__global__ void k_gj_pivot(double* A, int n, int p, int* perm, double* f, int* info) {
    __shared__ double sval[1024];
    __shared__ int sidx[1024];
    double best = -1.0;
    int bi = p;
    for (int i = p + threadIdx.x; i < n; i += blockDim.x) {
        const double v = fabs(A[(int64_t)i * n + p]);
        if (v > best) { best = v; bi = i; }
    }
    sval[threadIdx.x] = best;
    sidx[threadIdx.x] = bi;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            const double o = sval[threadIdx.x + w];
            const int oi = sidx[threadIdx.x + w];
            if (o > sval[threadIdx.x] || (o == sval[threadIdx.x] && oi < sidx[threadIdx.x])) {
                sval[threadIdx.x] = o;
                sidx[threadIdx.x] = oi;
            }
        }
        __syncthreads();
    }
    const int r = sidx[0];
    if (threadIdx.x == 0) perm[p] = r;
    if (r != p)
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            const double t = A[(int64_t)p * n + j];
            A[(int64_t)p * n + j] = A[(int64_t)r * n + j];
            A[(int64_t)r * n + j] = t;
        }
    __syncthreads();
    const double piv = A[(int64_t)p * n + p];
    if (piv == 0.0) {
        if (threadIdx.x == 0) *info = 1;
        return;
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) f[i] = (i == p) ? 0.0 : A[(int64_t)i * n + p];
    __syncthreads();
    const double inv = 1.0 / piv;
    for (int j = threadIdx.x; j < n; j += blockDim.x) A[(int64_t)p * n + j] = (j == p) ? inv : A[(int64_t)p * n + j] * inv;
}

__global__ void k_gj_eliminate(double* A, int n, int p, const double* f) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (j >= n || i == p) return;
    const double fi = f[i];
    if (fi == 0.0) return;
    const double apj = A[(int64_t)p * n + j];
    if (j == p) A[(int64_t)i * n + p] = -fi * apj;
    else A[(int64_t)i * n + j] -= fi * apj;
}

__global__ void k_swap_cols(double* A, int n, int a, int b) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double t = A[(int64_t)i * n + a];
    A[(int64_t)i * n + a] = A[(int64_t)i * n + b];
    A[(int64_t)i * n + b] = t;
}

int invert(cudaStream_t s, double* A, int n, double* work) {
    // work: n doubles (multipliers) + n ints (perm) + 1 int (info)
    double* f = work;
    int* perm = reinterpret_cast<int*>(work + n);
    int* info = perm + n;
    cudaMemsetAsync(info, 0, sizeof(int), s);
    dim3 eg((n + 255) / 256, n);
    for (int p = 0; p < n; ++p) {
        k_gj_pivot<<<1, 1024, 0, s>>>(A, n, p, perm, f, info);
        k_gj_eliminate<<<eg, 256, 0, s>>>(A, n, p, f);
    }
    std::vector<int> hp(n);
    int hinfo = 0;
    cudaMemcpyAsync(hp.data(), perm, sizeof(int) * n, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    if (hinfo) return 1;
    for (int p = n - 1; p >= 0; --p)
        if (hp[p] != p) k_swap_cols<<<(n + 255) / 256, 256, 0, s>>>(A, n, p, hp[p]);
    return 0;
}

// ---------------------------------------------------------------- elementwise helpers
__global__ void k_identity(double* A, int n, double scale) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)n * n) return;
    A[i] = (i / n == i % n) ? scale : 0.0;
}
void fill_identity(cudaStream_t s, double* A, int n, double scale) {
    k_identity<<<(unsigned)(((int64_t)n * n + 255) / 256), 256, 0, s>>>(A, n, scale);
}

__global__ void k_axpby(int64_t n, double a, const double* x, double b, double* y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = a * x[i] + b * y[i];
}
void axpby(cudaStream_t s, int64_t n, double a, const double* x, double b, double* y) {
    k_axpby<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, a, x, b, y);
}

__global__ void k_cast32(const double* in, float* out, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)in[i];
}
void cast_f64_f32(cudaStream_t s, const double* in, float* out, int64_t n) {
    k_cast32<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in, out, n);
}

// hi = bf16(x), lo = bf16(x - hi): x = hi + lo + O(2^-17 |x|)
__global__ void k_split(const double* in, __nv_bfloat16* hi, __nv_bfloat16* lo, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float x = (float)in[i];
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    hi[i] = h;
    lo[i] = __float2bfloat16_rn((float)(in[i] - (double)__bfloat162float(h)));
}
void split_bf16(cudaStream_t s, const double* in, void* hi, void* lo, int64_t n) {
    k_split<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in, (__nv_bfloat16*)hi, (__nv_bfloat16*)lo, n);
}

__global__ void k_transpose(const double* in, double* out, int rows, int cols) {
    __shared__ double tile[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int j = threadIdx.y; j < 32; j += 8) {
        const int r = by + j, c = bx + threadIdx.x;
        if (r < rows && c < cols) tile[j][threadIdx.x] = in[(int64_t)r * cols + c];
    }
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += 8) {
        const int r = bx + j, c = by + threadIdx.x;
        if (r < cols && c < rows) out[(int64_t)r * rows + c] = tile[threadIdx.x][j];
    }
}
void transpose(cudaStream_t s, const double* in, double* out, int rows, int cols) {
    dim3 g((cols + 31) / 32, (rows + 31) / 32), b(32, 8);
    k_transpose<<<g, b, 0, s>>>(in, out, rows, cols);
}

void scatter_incidence_dense(cudaStream_t, const int*, int, int, double*) {}

}  // namespace tdc
