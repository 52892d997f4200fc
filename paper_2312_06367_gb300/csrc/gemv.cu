// Stand-alone history sum of the MOT recurrence (Sec. IV-B) on caller-held blocks:
//   out[r][i] = sum_{q < nblk} sum_{j < n} blocks[q][i][j] x[q][r][j]
// One warp per (row i, block q) writes the per-block partial sums; a second kernel adds the
// blocks in a fixed order (deterministic result).
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "internal.h"

namespace tdc {

template <typename T, int RMAX>
__global__ void k_bg_partial(const T* __restrict__ blocks, int64_t nblk, int64_t n, const T* __restrict__ x, int R,
                             T* __restrict__ partial) {
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t q = blockIdx.y;
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    const T* a = blocks + (q * n + row) * n;
    const T* xq = x + q * R * n;
    T s[RMAX];
#pragma unroll
    for (int r = 0; r < RMAX; ++r) s[r] = 0;
    for (int64_t j = lane; j < n; j += 32) {
        const T v = a[j];
#pragma unroll
        for (int r = 0; r < RMAX; ++r)
            if (r < R) s[r] += v * xq[(int64_t)r * n + j];
    }
#pragma unroll
    for (int r = 0; r < RMAX; ++r) {
        T v = s[r];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0 && r < R) partial[(q * R + r) * n + row] = v;
    }
}

template <typename T>
__global__ void k_bg_reduce(const T* __restrict__ partial, int64_t nblk, int64_t n, int R, T* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * R) return;
    T s = 0;
    for (int64_t q = 0; q < nblk; ++q) s += partial[q * R * n + i];
    out[i] = s;
}

template <typename T>
static cudaError_t launch_block_gemv(const T* blocks, int64_t nblk, int64_t n, const T* x, int R, T* out, T* partial,
                                     cudaStream_t s) {
    const int wpb = 8;
    const dim3 g((unsigned)((n + wpb - 1) / wpb), (unsigned)nblk);
    if (R == 1) k_bg_partial<T, 1><<<g, 32 * wpb, 0, s>>>(blocks, nblk, n, x, R, partial);
    else if (R <= 4) k_bg_partial<T, 4><<<g, 32 * wpb, 0, s>>>(blocks, nblk, n, x, R, partial);
    else k_bg_partial<T, 8><<<g, 32 * wpb, 0, s>>>(blocks, nblk, n, x, R, partial);
    k_bg_reduce<T><<<(unsigned)((n * R + 255) / 256), 256, 0, s>>>(partial, nblk, n, R, out);
    return cudaGetLastError();
}

// common argument checks; returns 0 when the call may proceed
static tdcfie_status check_gemv(int precision, const void* blocks, int64_t nblk, int64_t n, const void* x, int64_t R,
                                void* out) {
    if (precision != TDCFIE_FP64 && precision != TDCFIE_FP32)
        return fail(nullptr, TDCFIE_E_UNSUPPORTED, "block GEMV supports TDCFIE_FP64 and TDCFIE_FP32");
    if (!blocks || !x || !out) return fail(nullptr, TDCFIE_E_ARG, "NULL device pointer");
    if (nblk < 1 || nblk > 65535 || n < 1 || n > (1 << 24) || R < 1 || R > 8)
        return fail(nullptr, TDCFIE_E_ARG, "sizes out of range (1 <= nblk <= 65535, 1 <= n <= 2^24, 1 <= R <= 8)");
    return TDCFIE_OK;
}

}  // namespace tdc

using namespace tdc;

extern "C" tdcfie_status tdcfie_block_gemv(int precision, const void* blocks, int64_t nblk, int64_t n, const void* x,
                                           int64_t R, void* out, void* stream) {
    tdcfie_status st = check_gemv(precision, blocks, nblk, n, x, R, out);
    if (st != TDCFIE_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t es = precision == TDCFIE_FP64 ? 8 : 4;
    void* partial = nullptr;
    cudaError_t e = cudaMallocAsync(&partial, es * (size_t)nblk * R * n, s);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaMallocAsync (block GEMV scratch)");
    if (precision == TDCFIE_FP64)
        e = launch_block_gemv<double>((const double*)blocks, nblk, n, (const double*)x, (int)R, (double*)out,
                                      (double*)partial, s);
    else
        e = launch_block_gemv<float>((const float*)blocks, nblk, n, (const float*)x, (int)R, (float*)out,
                                     (float*)partial, s);
    cudaError_t e2 = cudaFreeAsync(partial, s);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "block GEMV launch");
    if (e2 != cudaSuccess) return cuda_fail(nullptr, e2, "cudaFreeAsync (block GEMV scratch)");
    return TDCFIE_OK;
}

// ---------------------------------------------------------------- variant without allocation
// Some callers cannot allocate device memory when they need this sum: a thread of a process in
// which another thread holds a global-mode stream capture (cudaMalloc is not permitted then),
// services whose caching allocator has reserved nearly all of the HBM up front, or loops that
// cannot take the implicit synchronisation of an allocation.  For them the per-block partial sums
// live in this file-scope device array.  Every GPU that loads the library holds it (32 MiB) until
// the process exits.  In host code the name below is only a host-side stand-in for the array;
// the kernels receive the device address obtained with cudaGetSymbolAddress.
namespace tdc {
constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(32) << 20;
static __device__ __align__(256) unsigned char g_block_gemv_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 64;
static void* g_scratch_addr[NOALLOC_MAX_DEVICES];
static CUcontext g_scratch_ctx[NOALLOC_MAX_DEVICES];
static std::mutex g_scratch_mu;

// cuCtxGetCurrent through the runtime's driver entry point, so that the library keeps no link-time
// dependency on the driver library (it loads on hosts without a GPU)
typedef CUresult (*CtxGetCurrent)(CUcontext*);
static CtxGetCurrent ctx_get_current() {
    static CtxGetCurrent fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (CtxGetCurrent)p;
    }
    return fn;
}

// device address of the scratch array on the current device, looked up once per device and
// context (a cudaDeviceReset gives the device a new primary context and the array a new address)
static cudaError_t scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
    // no allocation and no synchronising call here: cudaGetDevice and cuCtxGetCurrent only, and
    // the symbol lookup (which also makes the primary context current) when the context is new
    const CtxGetCurrent get = ctx_get_current();
    if (!get) return cudaErrorDeviceUninitialized;
    CUcontext ctx = nullptr;
    if (get(&ctx) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev] || !ctx || g_scratch_ctx[dev] != ctx) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_block_gemv_scratch);
        if (e != cudaSuccess) return e;
        if (get(&ctx) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
        g_scratch_addr[dev] = p;
        g_scratch_ctx[dev] = ctx;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}
}  // namespace tdc

extern "C" tdcfie_status tdcfie_block_gemv_noalloc(int precision, const void* blocks, int64_t nblk, int64_t n,
                                                   const void* x, int64_t R, void* out, void* stream) {
    tdcfie_status st = check_gemv(precision, blocks, nblk, n, x, R, out);
    if (st != TDCFIE_OK) return st;
    const size_t es = precision == TDCFIE_FP64 ? 8 : 4;
    const double need = (double)es * (double)nblk * (double)R * (double)n;
    if (need > (double)NOALLOC_SCRATCH_BYTES)
        return fail(nullptr, TDCFIE_E_ARG,
                    "tdcfie_block_gemv_noalloc: nblk * R * n * element size exceeds the 32 MiB static scratch "
                    "(at most 4194304 FP64 or 8388608 FP32 partial sums); use tdcfie_block_gemv");
    void* partial = nullptr;
    cudaError_t e = scratch_address(&partial);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetSymbolAddress (static block GEMV scratch)");
    cudaStream_t s = (cudaStream_t)stream;
    if (precision == TDCFIE_FP64)
        e = launch_block_gemv<double>((const double*)blocks, nblk, n, (const double*)x, (int)R, (double*)out,
                                      (double*)partial, s);
    else
        e = launch_block_gemv<float>((const float*)blocks, nblk, n, (const float*)x, (int)R, (float*)out,
                                     (float*)partial, s);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "block GEMV launch");
    return TDCFIE_OK;
}
