// Far field of marched currents at one frequency (Sec. V: the large-time-step test compares the
// sphere's far field at 3 Hz with the series solution).  FP64 throughout; post-processing, not
// part of the step.
//
// Units c = eta = mu = 1, phasors e^{j w t}, k = w.  The march's j_i are hat-basis coefficients
// (Eq. post_processing) at t_i = i dt, whose spectrum is dt sinc^2(w dt / 2) e^{-j w t_i}:
//   J_m(w) = dt sinc^2(w dt / 2) sum_i j_m[i] e^{-j w t_i}
//   N(rhat) = sum_m J_m(w) int f_m(r) e^{j k rhat.r} dS       (7-point rule per triangle)
//   F(rhat) = -j k / (4 pi) (I - rhat rhat) N(rhat)           (scattered field = F e^{-j k r} / r)
// On triangle c the RWG function of the edge opposite local vertex q is
// tsign[c][q] (r - V[F[c][q]]) / (2 A_c) (Sec. II-C, Fig. 1).
#include <cmath>
#include <vector>

#include "internal.h"

namespace tdc {

struct Rule7 { double p[7][4]; };

// J[r][m] = sum_i ph[i] j[i][r][m]  (ph = dt sinc^2 e^{-j w t_i}, complex)
template <typename T>
__global__ void k_ff_spectrum(const T* __restrict__ j, int64_t nt, int R, int ne, const double2* __restrict__ ph,
                              double2* __restrict__ J) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)R * ne) return;
    double re = 0.0, im = 0.0;
    for (int64_t i = 0; i < nt; ++i) {
        const double v = (double)j[i * R * ne + t];
        re = fma(ph[i].x, v, re);
        im = fma(ph[i].y, v, im);
    }
    J[t] = make_double2(re, im);
}

// one block per (direction, wave): N summed over triangles, reduced in a fixed order
__global__ void __launch_bounds__(256) k_ff_sum(DevMesh m, Rule7 rule, double k, const double* __restrict__ rhat,
                                                const double2* __restrict__ J, int R, double* __restrict__ out) {
    const int d = blockIdx.x, r = blockIdx.y;
    const double ux = rhat[3 * d], uy = rhat[3 * d + 1], uz = rhat[3 * d + 2];
    double acc[6] = {0, 0, 0, 0, 0, 0};   // N: (re, im) of x, y, z
    for (int c = threadIdx.x; c < m.nc; c += blockDim.x) {
        const double* v0 = m.V + 3 * m.F[3 * c];
        const double* v1 = m.V + 3 * m.F[3 * c + 1];
        const double* v2 = m.V + 3 * m.F[3 * c + 2];
        const double ex = v1[0] - v0[0], ey = v1[1] - v0[1], ez = v1[2] - v0[2];
        const double fx = v2[0] - v0[0], fy = v2[1] - v0[1], fz = v2[2] - v0[2];
        const double nx = ey * fz - ez * fy, ny = ez * fx - ex * fz, nz = ex * fy - ey * fx;
        const double A = 0.5 * sqrt(nx * nx + ny * ny + nz * nz);
        // Q = int_c e^{j k u.x} (x - x0) dS and P = int_c e^{j k u.x} dS, so that
        // int_c e^{j k u.x} (x - V_q) dS = Q - (V_q - v0) P
        double Qr[3] = {0, 0, 0}, Qi[3] = {0, 0, 0}, Pr = 0.0, Pi = 0.0;
        for (int q = 0; q < 7; ++q) {
            const double a = rule.p[q][0], b = rule.p[q][1], cc = rule.p[q][2], w = rule.p[q][3] * A;
            const double x = a * v0[0] + b * v1[0] + cc * v2[0];
            const double y = a * v0[1] + b * v1[1] + cc * v2[1];
            const double z = a * v0[2] + b * v1[2] + cc * v2[2];
            double sn, cs;
            sincos(k * (ux * x + uy * y + uz * z), &sn, &cs);
            Pr = fma(w, cs, Pr);
            Pi = fma(w, sn, Pi);
            const double rel[3] = {x - v0[0], y - v0[1], z - v0[2]};
            for (int e = 0; e < 3; ++e) {
                Qr[e] = fma(w * cs, rel[e], Qr[e]);
                Qi[e] = fma(w * sn, rel[e], Qi[e]);
            }
        }
        for (int q = 0; q < 3; ++q) {
            const int mm = m.tedge[3 * c + q];
            const double* vq = m.V + 3 * m.F[3 * c + q];
            const double s = m.tsign[3 * c + q] / (2.0 * A);
            const double2 Jm = J[(int64_t)r * m.ne + mm];
            for (int e = 0; e < 3; ++e) {
                const double off = vq[e] - v0[e];
                const double ir = s * (Qr[e] - off * Pr), ii = s * (Qi[e] - off * Pi);   // int f_m e^{..} (component e)
                acc[2 * e] += Jm.x * ir - Jm.y * ii;
                acc[2 * e + 1] += Jm.x * ii + Jm.y * ir;
            }
        }
    }
    __shared__ double red[256 / 32][6];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int e = 0; e < 6; ++e) {
        double v = acc[e];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][e] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double N[6] = {0, 0, 0, 0, 0, 0};
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
            for (int e = 0; e < 6; ++e) N[e] += red[w][e];
        // F = -j k / (4 pi) (N - u (u.N))
        const double u[3] = {ux, uy, uz};
        const double dr = ux * N[0] + uy * N[2] + uz * N[4], di = ux * N[1] + uy * N[3] + uz * N[5];
        const double f = k / (4.0 * M_PI);
        for (int e = 0; e < 3; ++e) {
            const double pr = N[2 * e] - u[e] * dr, pi = N[2 * e + 1] - u[e] * di;
            double* o = out + ((int64_t)d * R + r) * 6 + 2 * e;
            o[0] = f * pi;      // -j f (pr + j pi) = f pi - j f pr
            o[1] = -f * pr;
        }
    }
}

tdcfie_status far_field(tdcfie_t h, const void* currents, int64_t nt, double w, const double* rhat, int64_t ndir,
                        double* out) {
    const int R = (int)h->R, ne = h->mesh.ne;
    cudaStream_t s = h->stream;
    const bool f64 = h->opts.precision == TDCFIE_FP64;
    // phase table: dt sinc^2(w dt / 2) e^{-j w t_i}
    const double dt = h->dt, x = 0.5 * w * dt;
    const double hat = x != 0.0 ? dt * (std::sin(x) / x) * (std::sin(x) / x) : dt;
    std::vector<double> ph(2 * nt);
    for (int64_t i = 0; i < nt; ++i) {
        const double t = (double)(i + 1) * dt;
        ph[2 * i] = hat * std::cos(w * t);
        ph[2 * i + 1] = -hat * std::sin(w * t);
    }
    Rule7 rule;
    triangle_rule7(rule.p);
    double *dph = nullptr, *dJ = nullptr, *drh = nullptr, *dout = nullptr;
    cudaError_t e = cudaMalloc(&dph, sizeof(double) * 2 * std::max<int64_t>(nt, 1));
    if (e == cudaSuccess) e = cudaMalloc(&dJ, sizeof(double) * 2 * R * ne);
    if (e == cudaSuccess) e = cudaMalloc(&drh, sizeof(double) * 3 * ndir);
    if (e == cudaSuccess) e = cudaMalloc(&dout, sizeof(double) * 6 * R * ndir);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dph, ph.data(), sizeof(double) * 2 * nt, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(drh, rhat, sizeof(double) * 3 * ndir, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        const unsigned g = (unsigned)(((int64_t)R * ne + 255) / 256);
        if (f64) k_ff_spectrum<double><<<g, 256, 0, s>>>((const double*)currents, nt, R, ne, (const double2*)dph, (double2*)dJ);
        else k_ff_spectrum<float><<<g, 256, 0, s>>>((const float*)currents, nt, R, ne, (const double2*)dph, (double2*)dJ);
        k_ff_sum<<<dim3((unsigned)ndir, (unsigned)R), 256, 0, s>>>(h->dm, rule, w, drh, (const double2*)dJ, R, dout);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, dout, sizeof(double) * 6 * R * ndir, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    for (void* p : {(void*)dph, (void*)dJ, (void*)drh, (void*)dout}) if (p) cudaFree(p);
    if (e != cudaSuccess) return cuda_fail(h, e, "far field");
    return TDCFIE_OK;
}

}  // namespace tdc
