// Device arithmetic of the SIMT (FP64 / FP32) step, shared by the per-handle step kernels
// (march.cu) and the persistent uneven-batch kernel (batch.cu), so that both compute the same
// values bit for bit.
#pragma once
#include "internal.h"

namespace tdc {

// ---------------------------------------------------------------- plane-wave tests
// Per edge m a list of quadrature points with a weighted basis vector: 7 points on each
// triangle of f_m (degree-5 rule, coefficient w A f_m(x)) for e_m and 3 points on each fine
// triangle of g_m (degree-2 rule, coefficient w A g_m(x)) for h_m.  Per step n and wave P:
//   e_m = sum_x c(x).p env(x, t_n),  h_m = sum_x c(x).(k x p) env(x, t_n),
//   env(x, t) = amp exp(-((t - k.x - t0)/width)^2).
template <typename T>
__device__ __forceinline__ T mul_rn(T a, T b);
template <>
__device__ __forceinline__ float mul_rn<float>(float a, float b) { return __fmul_rn(a, b); }
template <>
__device__ __forceinline__ double mul_rn<double>(double a, double b) { return __dmul_rn(a, b); }
template <typename T>
__device__ __forceinline__ T add_rn(T a, T b);
template <>
__device__ __forceinline__ float add_rn<float>(float a, float b) { return __fadd_rn(a, b); }
template <>
__device__ __forceinline__ double add_rn<double>(double a, double b) { return __dadd_rn(a, b); }

// Every multiply-add below is spelled out (fma or a rounded product), so that the per-handle
// kernels and the persistent batch kernel, which inline this code into different kernels, round
// identically.
template <typename T>
__device__ __forceinline__ void rhs_edge(const double* P, int64_t n, double dt, int mm, const int* __restrict__ pptr,
                                         const T* __restrict__ px, const T* __restrict__ pc, const int* __restrict__ nE,
                                         T& e_out, T& h_out) {
    const T kx = (T)P[0], ky = (T)P[1], kz = (T)P[2], qx = (T)P[3], qy = (T)P[4], qz = (T)P[5];
    const T amp = (T)P[6], inv_w = (T)(1.0 / P[8]);
    const T tt = (T)((double)n * dt - P[7]);
    const T hx = fma(ky, qz, -mul_rn(kz, qy)), hy = fma(kz, qx, -mul_rn(kx, qz)), hz = fma(kx, qy, -mul_rn(ky, qx));   // k x p
    T e = 0, h = 0;
    const int b = pptr[mm], me = b + nE[mm], end = pptr[mm + 1];
    for (int q = b; q < end; ++q) {
        const T x = px[3 * q], y = px[3 * q + 1], z = px[3 * q + 2];
        const T arg = mul_rn(add_rn(tt, -fma(kx, x, fma(ky, y, mul_rn(kz, z)))), inv_w);
        const T env = mul_rn(amp, exp(-mul_rn(arg, arg)));
        const T cx = pc[3 * q], cy = pc[3 * q + 1], cz = pc[3 * q + 2];
        if (q < me) e = fma(env, fma(cx, qx, fma(cy, qy, mul_rn(cz, qz))), e);
        else h = fma(env, fma(cx, hx, fma(cy, hy, mul_rn(cz, hz))), h);
    }
    e_out = e;
    h_out = h;
}

// ---------------------------------------------------------------- row dot products (SIMT)
// partial[q][r][i] = sum_j B_q[i][j] x_q[r][j] for one warp per (row i, block q); x_q is e_n, h_n
// or a ring slot chosen from the device step counter.
template <typename T> struct Vec2;
template <> struct Vec2<double> { using type = double2; };
template <> struct Vec2<float> { using type = float4; };

// Row dot products of one warp: acc[r] = B . x_r.  FP64: plain FP64 accumulation.  FP32: the
// products and their sums are carried error-free (each product's rounding error from an FMA, each
// addition's from Knuth's TwoSum), so the result equals the exact dot product of the FP32 inputs to
// about FP32 precision squared; the lanes are combined in FP64.  The MOT recurrence turns y into the
// current through (y_n - y_{n-1}) / dtt (Eq. post_processing), which magnifies any per-step error of
// y by about |y| / |y_n - y_{n-1}|; plain FP32 accumulation over rows of thousands of entries is
// then far above the reduced-precision bar at small time steps.
template <typename T, int RMAX>
struct RowDot {
    __device__ static void run(const T* __restrict__ B, int ncols, const T* __restrict__ x, int R, int ldx,
                               double* acc) {
        const int lane = threadIdx.x & 31;
        T s[RMAX];
#pragma unroll
        for (int r = 0; r < RMAX; ++r) s[r] = 0;
        for (int j = lane; j < ncols; j += 32) {
            const T a = B[j];
#pragma unroll
            for (int r = 0; r < RMAX; ++r)
                if (r < R) s[r] = fma(a, x[(int64_t)r * ldx + j], s[r]);
        }
#pragma unroll
        for (int r = 0; r < RMAX; ++r) {
            double v = (double)s[r];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            acc[r] = v;
        }
    }
};

__device__ __forceinline__ void ff_add(float& hi, float& lo, float a, float b) {
    // rounded operations only: a contracted multiply-add here would break the error-free sums
    const float p = __fmul_rn(a, b);
    const float pe = fmaf(a, b, -p);        // a b = p + pe exactly
    const float t = __fadd_rn(hi, p);        // TwoSum(hi, p) = t + te
    const float bp = __fsub_rn(t, hi);
    const float te = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bp)), __fsub_rn(p, bp));
    hi = t;
    lo = __fadd_rn(lo, __fadd_rn(te, pe));
}

template <int RMAX>
struct RowDot<float, RMAX> {
    __device__ static void run(const float* __restrict__ B, int ncols, const float* __restrict__ x, int R, int ldx,
                               double* acc) {
        const int lane = threadIdx.x & 31;
        // four independent compensated accumulators per right-hand side (one per float4 component)
        float hi[RMAX][4], lo[RMAX][4];
#pragma unroll
        for (int r = 0; r < RMAX; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) hi[r][c] = lo[r][c] = 0.f;
        const bool vec = ((ncols | ldx) & 3) == 0 && ((reinterpret_cast<uintptr_t>(B) | reinterpret_cast<uintptr_t>(x)) & 15) == 0;
        if (vec) {
            const float4* B4 = reinterpret_cast<const float4*>(B);
            for (int j = lane; j < (ncols >> 2); j += 32) {
                const float4 a = B4[j];
#pragma unroll
                for (int r = 0; r < RMAX; ++r)
                    if (r < R) {
                        const float4 v = reinterpret_cast<const float4*>(x + (int64_t)r * ldx)[j];
                        ff_add(hi[r][0], lo[r][0], a.x, v.x);
                        ff_add(hi[r][1], lo[r][1], a.y, v.y);
                        ff_add(hi[r][2], lo[r][2], a.z, v.z);
                        ff_add(hi[r][3], lo[r][3], a.w, v.w);
                    }
            }
        } else {
            for (int j = lane; j < ncols; j += 32) {
                const float a = B[j];
#pragma unroll
                for (int r = 0; r < RMAX; ++r)
                    if (r < R) ff_add(hi[r][0], lo[r][0], a, x[(int64_t)r * ldx + j]);
            }
        }
#pragma unroll
        for (int r = 0; r < RMAX; ++r) {
            double v = 0.0;
#pragma unroll
            for (int c = 0; c < 4; ++c) v += (double)hi[r][c] + (double)lo[r][c];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            acc[r] = v;
        }
    }
};

template <typename T, int RMAX>
__device__ __forceinline__ void warp_rows(const T* __restrict__ B, int ncols, const T* __restrict__ x, int R,
                                          int ldx, double* acc) {
    RowDot<T, RMAX>::run(B, ncols, x, R, ldx, acc);
}

// z_c = sum_j tsign[c][j] w[tedge[c][j]], w = (1/dtt - 1) y_n - y_{n-1}/dtt (y_{n-1} = 0 at n = 1)
template <typename T>
__device__ __forceinline__ double project_in_value(const DevMesh& m, int c, const T* __restrict__ yn,
                                                   const T* __restrict__ yp, bool first, double dtt) {
    double s = 0.0;
    for (int j = 0; j < 3; ++j) {
        const int e = m.tedge[3 * c + j];
        const double w = fma(1.0 / dtt - 1.0, (double)yn[e], -((first ? 0.0 : (double)yp[e]) / dtt));
        s = fma(m.tsign[3 * c + j], w, s);
    }
    return s;
}

}  // namespace tdc
