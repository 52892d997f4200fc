// FP64 device assembly of the space-time matrices (Sec. II-A..C, IV-A), natural units c = eta = 1.
//
//   S_k[m,n]    = -int int f_m(x).f_n(y) hdot_0(k dt - R) / (4 pi R)
//   Phi_k[c,c'] = -T0/(A_c A_c') int_c int_c' q_0(k dt - R) / (4 pi R)
//   MM_k[m,n]   =  int int g_m(x).[Rhat x f_n(y)] (h_0(k dt - R)/(4 pi R^2) + hdot_0(k dt - R)/(4 pi R))
//   Zs[m,n]     = -kappa int int g_m.g_n exp(-kappa R)/(4 pi R)
//   Psi[v,v']   = -(1/kappa) int int rho_v rho_v' exp(-kappa R)/(4 pi R),  rho_v = 1/(2 N_v A_t) on D_v
//   M[m,n]      =  int int g_m.[Rhat x f_n] (1 + kappa R) exp(-kappa R)/(4 pi R^2)
//   G[m,n]      =  int (n x g_m).f_n
//
// Quadrature rule (same rule as the reference implementation it is checked against):
//   outer: 7-point degree-5 rule on coarse triangles, 3-point degree-2 rule on fine triangles;
//   inner: polar decomposition about the projection of the outer point on the source plane,
//     one signed sub-triangle per edge, angular variable psi = asinh(lambda/h) split where the
//     breakpoint circles R = j dt cross the edge and into pieces of width <= 1, radial variable
//     u = asinh(rho/|d|) (rho when the pair is coplanar) split at the breakpoint radii and into
//     pieces of width <= 1; NANG and NRAD Gauss-Legendre points per piece;
//   retarded pairs other than a triangle with itself, when the projection p is well outside the
//     source triangle (every vertex at least two longest edges from p): polar coordinates about
//     p over the triangle's own angular range only (two halves split at the middle vertex, angle
//     variable psi = asinh(tan(theta - theta_f)) along the nearer boundary edge, split where
//     breakpoint circles cross a boundary edge and into pieces of width <= 1), radius from the
//     near to the far edge (split at breakpoint radii, u pieces of width <= 1); otherwise the
//     signed sub-triangle form above;
//   static pairs whose coarse parents share no vertex: 3 x 3 (fine-fine) and 3 x 7 (fine-coarse)
//     product rules; same-parent pairs are coplanar (d = 0) and the curl kernel vanishes there.
// Scatter: FP64 atomicAdd (order of summation is not fixed; results agree to rounding).
#include <cmath>
#include <cstdio>

#include "internal.h"

namespace tdc {

constexpr int MAXB = 64;   // breakpoints per (outer point, source triangle)
__constant__ double c_ax[NANG], c_aw[NANG], c_rx[NRAD], c_rw[NRAD];
__constant__ double c_r7[7][4];   // barycentric a, b, c, weight
__constant__ double c_r3[3][4];

void triangle_rule7(double r7[7][4]) {
    const double s15 = std::sqrt(15.0);
    const double a1 = (9.0 - 2.0 * s15) / 21.0, b1 = (6.0 + s15) / 21.0, w1 = (155.0 + s15) / 1200.0;
    const double a2 = (9.0 + 2.0 * s15) / 21.0, b2 = (6.0 - s15) / 21.0, w2 = (155.0 - s15) / 1200.0;
    const double t[7][4] = {{1.0 / 3, 1.0 / 3, 1.0 / 3, 9.0 / 40.0},
                            {a1, b1, b1, w1}, {b1, a1, b1, w1}, {b1, b1, a1, w1},
                            {a2, b2, b2, w2}, {b2, a2, b2, w2}, {b2, b2, a2, w2}};
    for (int q = 0; q < 7; ++q)
        for (int c = 0; c < 4; ++c) r7[q][c] = t[q][c];
}

void set_rule_tables(const RuleTables& r, cudaStream_t s) {
    cudaMemcpyToSymbolAsync(c_ax, r.ax, sizeof(r.ax), 0, cudaMemcpyHostToDevice, s);
    cudaMemcpyToSymbolAsync(c_aw, r.aw, sizeof(r.aw), 0, cudaMemcpyHostToDevice, s);
    cudaMemcpyToSymbolAsync(c_rx, r.rx, sizeof(r.rx), 0, cudaMemcpyHostToDevice, s);
    cudaMemcpyToSymbolAsync(c_rw, r.rw, sizeof(r.rw), 0, cudaMemcpyHostToDevice, s);
    // symmetric rules: degree 5 (7 points) and degree 2 (3 points)
    double r7[7][4];
    triangle_rule7(r7);
    double r3[3][4] = {{2.0 / 3, 1.0 / 6, 1.0 / 6, 1.0 / 3}, {1.0 / 6, 2.0 / 3, 1.0 / 6, 1.0 / 3},
                       {1.0 / 6, 1.0 / 6, 2.0 / 3, 1.0 / 3}};
    cudaMemcpyToSymbolAsync(c_r7, r7, sizeof(r7), 0, cudaMemcpyHostToDevice, s);
    cudaMemcpyToSymbolAsync(c_r3, r3, sizeof(r3), 0, cudaMemcpyHostToDevice, s);
}

struct V3 { double x, y, z; };
__device__ __forceinline__ V3 mk(const double* p) { return {p[0], p[1], p[2]}; }
__device__ __forceinline__ V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ V3 operator*(double s, V3 a) { return {s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V3 cross(V3 a, V3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
__device__ __forceinline__ double nrm(V3 a) { return sqrt(dot(a, a)); }

// Temporal basis (Sec. IV-A).  Order 1: the hat h_0 on [-dt, dt] and the C1 quadratic q_0 on
// [-dt, 2 dt].  Order 2 (the remark closing Sec. IV-B): the shifted quadratic Lagrange
// interpolator, s = t / dt,
//   h_0 = (s+1)(s+2)/2 on [-1, 0),  1 - s^2 on [0, 1),  (s-1)(s-2)/2 on [1, 2],
// and q_0 with q_0' = (h_0(t) - h_0(t - dt)) / dt, zero before -dt: q_0(s) = H(s) - H(s - 1) with
// H(s) the integral of h_0 from -1 to s (q_0 vanishes again after 3 dt).
__constant__ int c_torder;

__device__ __forceinline__ double H2(double s) {
    if (s <= -1.0) return 0.0;
    if (s < 0.0) { const double u = s + 1.0; return u * u * u / 6.0 + u * u / 4.0; }
    if (s < 1.0) return 5.0 / 12.0 + s - s * s * s / 3.0;
    if (s < 2.0) { const double v = s - 1.0; return 13.0 / 12.0 + v * v * v / 6.0 - v * v / 4.0; }
    return 1.0;
}
__device__ __forceinline__ double h0f(double t, double dt) {
    if (c_torder == 2) {
        const double s = t / dt;
        if (s >= -1.0 && s < 0.0) return 0.5 * (s + 1.0) * (s + 2.0);
        if (s >= 0.0 && s < 1.0) return 1.0 - s * s;
        if (s >= 1.0 && s <= 2.0) return 0.5 * (s - 1.0) * (s - 2.0);
        return 0.0;
    }
    if (t >= -dt && t < 0.0) return 1.0 + t / dt;
    if (t >= 0.0 && t <= dt) return 1.0 - t / dt;
    return 0.0;
}
__device__ __forceinline__ double h0d(double t, double dt) {
    if (c_torder == 2) {
        const double s = t / dt;
        if (s > -1.0 && s < 0.0) return (s + 1.5) / dt;
        if (s > 0.0 && s < 1.0) return -2.0 * s / dt;
        if (s > 1.0 && s < 2.0) return (s - 1.5) / dt;
        return 0.0;
    }
    if (t > -dt && t < 0.0) return 1.0 / dt;
    if (t > 0.0 && t < dt) return -1.0 / dt;
    return 0.0;
}
__device__ __forceinline__ double q0f(double t, double dt) {
    const double s = t / dt;
    if (c_torder == 2) return H2(s) - H2(s - 1.0);
    if (t >= -dt && t < 0.0) return 0.5 * (s + 1.0) * (s + 1.0);
    if (t >= 0.0 && t < dt) return 0.5 - s * s + s;
    if (t >= dt && t <= 2.0 * dt) return 0.5 * (s - 2.0) * (s - 2.0);
    return 0.0;
}

__device__ __forceinline__ void sort_small(double* a, int n) {
    for (int i = 1; i < n; ++i) { double v = a[i]; int j = i - 1; while (j >= 0 && a[j] > v) { a[j + 1] = a[j]; --j; } a[j + 1] = v; }
}

// Polar rule over the source triangle (v0, v1, v2) for the outer point x.  For every inner node
// cb(R, W, y - x) is called; sum W * G(y) approximates int G dy.  brk: ascending breakpoint
// distances (only those that may cross the triangle).
template <class CB>
__device__ void polar(V3 x, V3 v0, V3 v1, V3 v2, const double* brk, int nb, bool coplanar, CB& cb) {
    V3 n = cross(v1 - v0, v2 - v0);
    n = (1.0 / nrm(n)) * n;
    const double d = coplanar ? 0.0 : dot(x - v0, n);
    const double ad = fabs(d);
    const V3 p = x - d * n;
    double rb[MAXB];
    int nrb = 0;
    for (int b = 0; b < nb; ++b)
        if (brk[b] > ad) rb[nrb++] = sqrt(brk[b] * brk[b] - d * d);
    const V3 vv[3] = {v0, v1, v2};
    for (int s = 0; s < 3; ++s) {
        const V3 a = vv[s], b = vv[(s + 1) % 3];
        const V3 ab = b - a;
        const double L = nrm(ab);
        const V3 e = (1.0 / L) * ab;
        double sig = dot(cross(a - p, b - p), n);
        if (sig == 0.0) continue;
        sig = sig > 0.0 ? 1.0 : -1.0;
        const double t = dot(p - a, e);
        const V3 f = a + t * e;
        V3 nu = f - p;
        const double h = nrm(nu);
        if (h <= 1e-14 * L) continue;
        nu = (1.0 / h) * nu;
        const double psa = asinh(-t / h), psb = asinh((L - t) / h);
        double sp[2 * MAXB + 2];
        int nsp = 0;
        sp[nsp++] = psa;
        for (int q = 0; q < nrb; ++q)
            if (rb[q] > h) {
                const double c = acosh(rb[q] / h);
                if (-c > psa && -c < psb) sp[nsp++] = -c;
                if (c > psa && c < psb) sp[nsp++] = c;
            }
        sp[nsp++] = psb;
        sort_small(sp, nsp);
        for (int pc = 0; pc + 1 < nsp; ++pc) {
            const double P0 = sp[pc], P1 = sp[pc + 1];
            if (P1 <= P0) continue;
            int nsub = (int)ceil((P1 - P0) / PIECE);
            if (nsub < 1) nsub = 1;
            const double hw = (P1 - P0) / nsub;
            for (int sb = 0; sb < nsub; ++sb) {
                const double q0 = P0 + sb * hw;
                for (int ga = 0; ga < NANG; ++ga) {
                    const double psi = q0 + 0.5 * hw * (c_ax[ga] + 1.0);
                    const double ch = cosh(psi), sh = sinh(psi);
                    const V3 om = (1.0 / ch) * (nu + sh * e);
                    const double rhoe = h * ch;
                    const double ang = sig * 0.5 * hw * c_aw[ga] / ch;
                    double rp[MAXB + 2];
                    int nrp = 0;
                    rp[nrp++] = 0.0;
                    for (int q = 0; q < nrb; ++q)
                        if (rb[q] > 0.0 && rb[q] < rhoe) rp[nrp++] = rb[q];
                    rp[nrp++] = rhoe;
                    sort_small(rp, nrp);
                    for (int ri = 0; ri + 1 < nrp; ++ri) {
                        const double r0 = rp[ri], r1 = rp[ri + 1];
                        if (r1 <= r0) continue;
                        if (ad > 0.0) {
                            const double u0 = asinh(r0 / ad), u1 = asinh(r1 / ad);
                            int ns = (int)ceil((u1 - u0) / PIECE);
                            if (ns < 1) ns = 1;
                            const double uw = (u1 - u0) / ns;
                            for (int k = 0; k < ns; ++k) {
                                const double ua = u0 + k * uw;
                                for (int gr = 0; gr < NRAD; ++gr) {
                                    const double u = ua + 0.5 * uw * (c_rx[gr] + 1.0);
                                    const double rho = ad * sinh(u), R = ad * cosh(u);
                                    const double W = ang * 0.5 * uw * c_rw[gr] * rho * R;
                                    cb(R, W, rho * om - d * n);
                                }
                            }
                        } else {
                            const double rw = r1 - r0;
                            for (int gr = 0; gr < NRAD; ++gr) {
                                const double rho = r0 + 0.5 * rw * (c_rx[gr] + 1.0);
                                cb(rho, ang * 0.5 * rw * c_rw[gr] * rho, rho * om);
                            }
                        }
                    }
                }
            }
        }
    }
}


__device__ __forceinline__ double cr2(double ax, double ay, double bx, double by) { return ax * by - ay * bx; }

// Far form: integrate over the triangle's own angular range seen from p (no signed cancellation).
template <class CB>
__device__ void polar_far(V3 x, V3 v0, V3 v1, V3 v2, const double* brk, int nb, CB& cb) {
    V3 n = cross(v1 - v0, v2 - v0);
    n = (1.0 / nrm(n)) * n;
    const double d = dot(x - v0, n), ad = fabs(d);
    const V3 p = x - d * n;
    const V3 vv[3] = {v0, v1, v2};
    bool inside = true;
    double lmax = 0.0, vmin = 1e300;
    for (int i = 0; i < 3; ++i) {
        if (dot(cross(vv[i] - p, vv[(i + 1) % 3] - p), n) < 0.0) inside = false;
        lmax = fmax(lmax, nrm(vv[(i + 1) % 3] - vv[i]));
        vmin = fmin(vmin, nrm(vv[i] - p));
    }
    if (inside || vmin < 2.0 * lmax) {
        polar(x, v0, v1, v2, brk, nb, false, cb);
        return;
    }
    V3 g = (1.0 / 3.0) * (v0 + v1 + v2) - p;
    const V3 u = (1.0 / nrm(g)) * g, w = cross(n, u);
    double X[3], Y[3], ph[3];
    for (int i = 0; i < 3; ++i) {
        X[i] = dot(vv[i] - p, u);
        Y[i] = dot(vv[i] - p, w);
        ph[i] = atan2(Y[i], X[i]);
    }
    int o[3] = {0, 1, 2};
    for (int i = 1; i < 3; ++i) { int t = o[i], j = i - 1; while (j >= 0 && ph[o[j]] > ph[t]) { o[j + 1] = o[j]; --j; } o[j + 1] = t; }
    const int L = o[0], Mv = o[1], H = o[2];
    double rb[MAXB];
    int nrb = 0;
    for (int b = 0; b < nb; ++b)
        if (brk[b] > ad) rb[nrb++] = sqrt(brk[b] * brk[b] - d * d);
    for (int half = 0; half < 2; ++half) {
        const double P0 = half == 0 ? ph[L] : ph[Mv], P1 = half == 0 ? ph[Mv] : ph[H];
        if (!(P1 > P0)) continue;
        const int ea[2] = {L, half == 0 ? L : Mv}, eb[2] = {H, half == 0 ? Mv : H};
        double re_mid[2];
        {
            const double th = 0.5 * (P0 + P1), c = cos(th), sn = sin(th);
            for (int ei = 0; ei < 2; ++ei) {
                const double ax = X[ea[ei]], ay = Y[ea[ei]], bx = X[eb[ei]], by = Y[eb[ei]];
                re_mid[ei] = cr2(ax, ay, bx - ax, by - ay) / cr2(c, sn, bx - ax, by - ay);
            }
        }
        const int en = re_mid[0] < re_mid[1] ? 0 : 1;
        const double nax = X[ea[en]], nay = Y[ea[en]], ndx = X[eb[en]] - nax, ndy = Y[eb[en]] - nay;
        const double tf = -(nax * ndx + nay * ndy) / (ndx * ndx + ndy * ndy);
        const double fx = nax + tf * ndx, fy = nay + tf * ndy;
        const double hn = sqrt(fx * fx + fy * fy);
        if (!(hn > 0.0)) continue;
        const double thf = atan2(fy, fx);
        double sp[4 * MAXB + 2];
        int nsp = 0;
        sp[nsp++] = P0;
        for (int ei = 0; ei < 2; ++ei) {
            const double ax = X[ea[ei]], ay = Y[ea[ei]], dx = X[eb[ei]] - ax, dy = Y[eb[ei]] - ay;
            const double dd = dx * dx + dy * dy;
            for (int q = 0; q < nrb; ++q) {
                const double bq = ax * dx + ay * dy, cq = ax * ax + ay * ay - rb[q] * rb[q];
                const double disc = bq * bq - dd * cq;
                if (disc <= 0.0) continue;
                const double sq = sqrt(disc);
                const double ts[2] = {(-bq - sq) / dd, (-bq + sq) / dd};
                for (int k = 0; k < 2; ++k) {
                    if (ts[k] <= 0.0 || ts[k] >= 1.0) continue;
                    const double ang = atan2(ay + ts[k] * dy, ax + ts[k] * dx);
                    if (ang > P0 && ang < P1) sp[nsp++] = ang;
                }
            }
        }
        sp[nsp++] = P1;
        sort_small(sp, nsp);
        for (int pc = 0; pc + 1 < nsp; ++pc) {
            const double S0 = asinh(tan(sp[pc] - thf)), S1 = asinh(tan(sp[pc + 1] - thf));
            if (!(S1 > S0)) continue;
            int nsub = (int)ceil((S1 - S0) / PIECE);
            if (nsub < 1) nsub = 1;
            const double hw = (S1 - S0) / nsub;
            for (int sb = 0; sb < nsub; ++sb) {
                for (int ga = 0; ga < NANG; ++ga) {
                    const double psi = S0 + sb * hw + 0.5 * hw * (c_ax[ga] + 1.0);
                    const double wth = 0.5 * hw * c_aw[ga] / cosh(psi);
                    const double th = thf + atan(sinh(psi));
                    const double c = cos(th), sn = sin(th);
                    double re[2];
                    for (int ei = 0; ei < 2; ++ei) {
                        const double ax = X[ea[ei]], ay = Y[ea[ei]], bx = X[eb[ei]], by = Y[eb[ei]];
                        re[ei] = cr2(ax, ay, bx - ax, by - ay) / cr2(c, sn, bx - ax, by - ay);
                    }
                    const double r0 = re[en], r1 = re[1 - en];
                    const V3 om = c * u + sn * w;
                    double rp[MAXB + 2];
                    int nrp = 0;
                    rp[nrp++] = r0;
                    for (int q = 0; q < nrb; ++q)
                        if (rb[q] > r0 && rb[q] < r1) rp[nrp++] = rb[q];
                    rp[nrp++] = r1;
                    sort_small(rp, nrp);
                    for (int ri = 0; ri + 1 < nrp; ++ri) {
                        const double a0 = rp[ri], a1 = rp[ri + 1];
                        if (!(a1 > a0)) continue;
                        if (ad > 0.0) {
                            const double u0 = asinh(a0 / ad), u1 = asinh(a1 / ad);
                            int ns = (int)ceil((u1 - u0) / PIECE);
                            if (ns < 1) ns = 1;
                            const double uw = (u1 - u0) / ns;
                            for (int k = 0; k < ns; ++k)
                                for (int gr = 0; gr < NRAD; ++gr) {
                                    const double uu = u0 + k * uw + 0.5 * uw * (c_rx[gr] + 1.0);
                                    const double rho = ad * sinh(uu), R = ad * cosh(uu);
                                    cb(R, wth * 0.5 * uw * c_rw[gr] * rho * R, rho * om - d * n);
                                }
                        } else {
                            const double rw = a1 - a0;
                            for (int gr = 0; gr < NRAD; ++gr) {
                                const double rho = a0 + 0.5 * rw * (c_rx[gr] + 1.0);
                                cb(rho, wth * 0.5 * rw * c_rw[gr] * rho, rho * om);
                            }
                        }
                    }
                }
            }
        }
    }
}

__device__ __forceinline__ V3 tri_pt(const double (*r)[4], int q, V3 a, V3 b, V3 c) {
    return r[q][0] * a + r[q][1] * b + r[q][2] * c;
}
__device__ __forceinline__ double tri_area(V3 a, V3 b, V3 c) { return 0.5 * nrm(cross(b - a, c - a)); }

// distance bounds from x to the triangle: lower = max(|d|, min vertex distance - longest edge);
// ad = |d|, the height of x over the source plane
__device__ __forceinline__ void dist_bounds(V3 x, V3 a, V3 b, V3 c, double& lo, double& hi, double& ad) {
    const double da = nrm(x - a), db = nrm(x - b), dc = nrm(x - c);
    const double L = fmax(nrm(b - a), fmax(nrm(c - b), nrm(a - c)));
    V3 n = cross(b - a, c - a);
    n = (1.0 / nrm(n)) * n;
    ad = fabs(dot(x - a, n));
    lo = fmax(ad, fmin(da, fmin(db, dc)) - L);
    lo = fmax(lo, 0.0);
    hi = fmax(da, fmax(db, dc));
}

// breakpoints j dt in (ad, hi]: every circle that can cross a signed sub-triangle (the
// sub-triangles start at the projection point, so radii below the triangle's own distance
// range still split their radial integrals)
__device__ __forceinline__ int make_breaks(double ad, double hi, double dt, double* brk, int* overflow) {
    int j0 = (int)floor(ad / dt);
    if (j0 < 1) j0 = 1;
    int nb = 0;
    for (int j = j0; j * dt <= hi + dt; ++j) {
        if (nb == MAXB) { atomicOr(overflow, 1); break; }
        brk[nb++] = j * dt;
    }
    return nb;
}

// ------------------------------------------------------------------ retarded EFIE
struct EfieAcc {
    double dt, T0;
    int k0;                 // first lag of the window
    int nk;                 // lags in the window
    double s0[LAGW], s1[LAGW][3], p0[LAGW];
    __device__ void operator()(double R, double W, V3 ymx) {
        for (int i = 0; i < nk; ++i) {
            const double tau = (k0 + i) * dt - R;
            if (tau <= -dt || tau >= (c_torder + 1) * dt) continue;      // support of q_0
            const double inv = 1.0 / (4.0 * M_PI * R);
            const double fs = -h0d(tau, dt) * inv;
            s0[i] += W * fs;
            s1[i][0] += W * fs * ymx.x; s1[i][1] += W * fs * ymx.y; s1[i][2] += W * fs * ymx.z;
            p0[i] += W * (-T0 * q0f(tau, dt) * inv);
        }
    }
};

__global__ void k_retarded_efie(DevMesh m, double dt, int K, double T0, double* __restrict__ S,
                                double* __restrict__ Phi, int* overflow) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)m.nc * 7 * m.nc;
    if (tid >= total) return;
    const int c2 = (int)(tid % m.nc);
    const int64_t rest = tid / m.nc;
    const int q = (int)(rest % 7);
    const int c = (int)(rest / 7);
    const V3 w0 = mk(m.V + 3 * m.F[3 * c]), w1 = mk(m.V + 3 * m.F[3 * c + 1]), w2 = mk(m.V + 3 * m.F[3 * c + 2]);
    const V3 v0 = mk(m.V + 3 * m.F[3 * c2]), v1 = mk(m.V + 3 * m.F[3 * c2 + 1]), v2 = mk(m.V + 3 * m.F[3 * c2 + 2]);
    const double A = tri_area(w0, w1, w2), A2 = tri_area(v0, v1, v2);
    const V3 x = tri_pt(c_r7, q, w0, w1, w2);
    const double wx = c_r7[q][3] * A;
    double lo, hi, ad;
    dist_bounds(x, v0, v1, v2, lo, hi, ad);
    double brk[MAXB];
    const int nb = make_breaks(ad, hi, dt, brk, overflow);
    int klo = (int)floor(lo / dt) - 1;
    if (klo < 0) klo = 0;
    int khi = (int)ceil(hi / dt) + c_torder + 1;
    if (khi > K - 1) khi = K - 1;
    const V3 wv[3] = {w0, w1, w2}, vv[3] = {v0, v1, v2};
    for (int k0 = klo; k0 <= khi; k0 += LAGW) {
        EfieAcc acc;
        acc.dt = dt; acc.T0 = T0; acc.k0 = k0;
        acc.nk = min(LAGW, khi - k0 + 1);
        for (int i = 0; i < LAGW; ++i) { acc.s0[i] = 0; acc.s1[i][0] = acc.s1[i][1] = acc.s1[i][2] = 0; acc.p0[i] = 0; }
        if (c == c2) polar(x, v0, v1, v2, brk, nb, true, acc);
        else polar_far(x, v0, v1, v2, brk, nb, acc);
        for (int i = 0; i < acc.nk; ++i) {
            const int k = k0 + i;
            atomicAdd(Phi + ((int64_t)k * m.nc + c) * m.nc + c2, wx * acc.p0[i] / (A * A2));
            if (acc.s0[i] == 0.0 && acc.s1[i][0] == 0.0 && acc.s1[i][1] == 0.0 && acc.s1[i][2] == 0.0) continue;
            const V3 s1 = {acc.s1[i][0], acc.s1[i][1], acc.s1[i][2]};
            for (int jj = 0; jj < 3; ++jj) {
                const V3 Iy = (m.tsign[3 * c2 + jj] / (2.0 * A2)) * (s1 + acc.s0[i] * (x - vv[jj]));
                const int n = m.tedge[3 * c2 + jj];
                for (int ii = 0; ii < 3; ++ii) {
                    const V3 Lx = (m.tsign[3 * c + ii] / (2.0 * A)) * (x - wv[ii]);
                    atomicAdd(S + ((int64_t)k * m.ne + m.tedge[3 * c + ii]) * m.ne + n, wx * dot(Lx, Iy));
                }
            }
        }
    }
}

// ------------------------------------------------------------------ retarded MFIE
struct MfieAcc {
    double dt;
    int k0, nk;
    double m1[LAGW][3];
    __device__ void operator()(double R, double W, V3 ymx) {
        for (int i = 0; i < nk; ++i) {
            const double tau = (k0 + i) * dt - R;
            if (tau <= -dt || tau >= c_torder * dt) continue;            // support of h_0
            const double fm = (h0f(tau, dt) / R + h0d(tau, dt)) / (4.0 * M_PI * R * R);
            m1[i][0] += W * fm * ymx.x; m1[i][1] += W * fm * ymx.y; m1[i][2] += W * fm * ymx.z;
        }
    }
};

__global__ void k_retarded_mfie(DevMesh m, double dt, int K, double* __restrict__ MM, int* overflow) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)m.nf * 3 * m.nc;
    if (tid >= total) return;
    const int c2 = (int)(tid % m.nc);
    const int64_t rest = tid / m.nc;
    const int q = (int)(rest % 3);
    const int t = (int)(rest / 3);
    if (m.fparent[t] == c2) return;   // coplanar: the curl kernel vanishes
    const V3 w0 = mk(m.fV + 3 * m.fF[3 * t]), w1 = mk(m.fV + 3 * m.fF[3 * t + 1]), w2 = mk(m.fV + 3 * m.fF[3 * t + 2]);
    const V3 v0 = mk(m.V + 3 * m.F[3 * c2]), v1 = mk(m.V + 3 * m.F[3 * c2 + 1]), v2 = mk(m.V + 3 * m.F[3 * c2 + 2]);
    const double A = tri_area(w0, w1, w2), A2 = tri_area(v0, v1, v2);
    const V3 x = tri_pt(c_r3, q, w0, w1, w2);
    const double wx = c_r3[q][3] * A;
    double lo, hi, ad;
    dist_bounds(x, v0, v1, v2, lo, hi, ad);
    double brk[MAXB];
    const int nb = make_breaks(ad, hi, dt, brk, overflow);
    int klo = (int)floor(lo / dt) - 1;
    if (klo < 0) klo = 0;
    int khi = (int)ceil(hi / dt) + c_torder + 1;
    if (khi > K - 1) khi = K - 1;
    const V3 wv[3] = {w0, w1, w2}, vv[3] = {v0, v1, v2};
    for (int k0 = klo; k0 <= khi; k0 += LAGW) {
        MfieAcc acc;
        acc.dt = dt; acc.k0 = k0; acc.nk = min(LAGW, khi - k0 + 1);
        for (int i = 0; i < LAGW; ++i) acc.m1[i][0] = acc.m1[i][1] = acc.m1[i][2] = 0.0;
        polar_far(x, v0, v1, v2, brk, nb, acc);
        for (int i = 0; i < acc.nk; ++i) {
            const V3 m1 = {acc.m1[i][0], acc.m1[i][1], acc.m1[i][2]};
            if (m1.x == 0.0 && m1.y == 0.0 && m1.z == 0.0) continue;
            const int k = k0 + i;
            double val[3][3];   // [local outer field i][inner edge jj]
            for (int jj = 0; jj < 3; ++jj) {
                const V3 cr = (m.tsign[3 * c2 + jj] / (2.0 * A2)) * cross(x - vv[jj], m1);
                for (int ii = 0; ii < 3; ++ii) val[ii][jj] = wx * dot((1.0 / (2.0 * A)) * (x - wv[ii]), cr);
            }
            for (int e = m.bc_ptr[t]; e < m.bc_ptr[t + 1]; ++e) {
                const int fn = m.bc_fn[e];
                const double* ph = m.bc_phi + 3 * e;
                for (int jj = 0; jj < 3; ++jj) {
                    const double v = ph[0] * val[0][jj] + ph[1] * val[1][jj] + ph[2] * val[2][jj];
                    if (v != 0.0) atomicAdd(MM + ((int64_t)k * m.ne + fn) * m.ne + m.tedge[3 * c2 + jj], v);
                }
            }
        }
    }
}

// ------------------------------------------------------------------ static matrices
struct YukAcc {
    double kappa;
    bool want_z, want_m;
    double z0; V3 z1; V3 mm1;
    __device__ void operator()(double R, double W, V3 ymx) {
        const double ek = exp(-kappa * R);
        if (want_z) {
            const double g = ek / (4.0 * M_PI * R);
            z0 += W * g;
            z1 = z1 + (W * g) * ymx;
        }
        if (want_m) {
            const double g = (1.0 + kappa * R) * ek / (4.0 * M_PI * R * R * R);
            mm1 = mm1 + (W * g) * ymx;
        }
    }
};

__device__ __forceinline__ bool parents_touch(const int* F, int a, int b) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            if (F[3 * a + i] == F[3 * b + j]) return true;
    return false;
}

// Zs and Psi: one thread per (outer fine triangle, inner fine triangle)
__global__ void k_static_efie(DevMesh m, double kappa, double* __restrict__ Zs, double* __restrict__ Psi) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)m.nf * m.nf;
    if (tid >= total) return;
    const int t2 = (int)(tid % m.nf), t = (int)(tid / m.nf);
    const V3 w[3] = {mk(m.fV + 3 * m.fF[3 * t]), mk(m.fV + 3 * m.fF[3 * t + 1]), mk(m.fV + 3 * m.fF[3 * t + 2])};
    const V3 v[3] = {mk(m.fV + 3 * m.fF[3 * t2]), mk(m.fV + 3 * m.fF[3 * t2 + 1]), mk(m.fV + 3 * m.fF[3 * t2 + 2])};
    const double A = tri_area(w[0], w[1], w[2]), A2 = tri_area(v[0], v[1], v[2]);
    const bool near = parents_touch(m.F, m.fparent[t], m.fparent[t2]);
    const bool copl = m.fparent[t] == m.fparent[t2];
    double I[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    double Is = 0.0;
    for (int q = 0; q < 3; ++q) {
        const V3 x = tri_pt(c_r3, q, w[0], w[1], w[2]);
        const double wx = c_r3[q][3] * A;
        double z0 = 0.0;
        V3 z1 = {0, 0, 0};
        if (near) {
            YukAcc acc{kappa, true, false, 0.0, {0, 0, 0}, {0, 0, 0}};
            polar(x, v[0], v[1], v[2], nullptr, 0, copl, acc);
            z0 = acc.z0; z1 = acc.z1;
        } else {
            for (int q2 = 0; q2 < 3; ++q2) {
                const V3 ymx = tri_pt(c_r3, q2, v[0], v[1], v[2]) - x;
                const double R = nrm(ymx);
                const double g = c_r3[q2][3] * A2 * exp(-kappa * R) / (4.0 * M_PI * R);
                z0 += g;
                z1 = z1 + g * ymx;
            }
        }
        Is += wx * z0;
        for (int j = 0; j < 3; ++j) {
            const V3 Iy = (1.0 / (2.0 * A2)) * (z1 + z0 * (x - v[j]));
            for (int i = 0; i < 3; ++i) I[i][j] += wx * dot((1.0 / (2.0 * A)) * (x - w[i]), Iy);
        }
    }
    const double rv = 1.0 / (2.0 * m.valence[m.fvert[t]] * A), rv2 = 1.0 / (2.0 * m.valence[m.fvert[t2]] * A2);
    atomicAdd(Psi + (int64_t)m.fvert[t] * m.nv + m.fvert[t2], -(1.0 / kappa) * rv * rv2 * Is);
    for (int e1 = m.bc_ptr[t]; e1 < m.bc_ptr[t + 1]; ++e1) {
        const double* p1 = m.bc_phi + 3 * e1;
        double u[3];
        for (int j = 0; j < 3; ++j) u[j] = p1[0] * I[0][j] + p1[1] * I[1][j] + p1[2] * I[2][j];
        for (int e2 = m.bc_ptr[t2]; e2 < m.bc_ptr[t2 + 1]; ++e2) {
            const double* p2 = m.bc_phi + 3 * e2;
            const double acc = p2[0] * u[0] + p2[1] * u[1] + p2[2] * u[2];
            atomicAdd(Zs + (int64_t)m.bc_fn[e1] * m.ne + m.bc_fn[e2], -kappa * acc);
        }
    }
}

// M: one thread per (outer fine triangle, inner coarse triangle)
__global__ void k_static_mfie(DevMesh m, double kappa, double* __restrict__ M) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)m.nf * m.nc;
    if (tid >= total) return;
    const int c2 = (int)(tid % m.nc), t = (int)(tid / m.nc);
    if (m.fparent[t] == c2) return;
    const V3 w[3] = {mk(m.fV + 3 * m.fF[3 * t]), mk(m.fV + 3 * m.fF[3 * t + 1]), mk(m.fV + 3 * m.fF[3 * t + 2])};
    const V3 v[3] = {mk(m.V + 3 * m.F[3 * c2]), mk(m.V + 3 * m.F[3 * c2 + 1]), mk(m.V + 3 * m.F[3 * c2 + 2])};
    const double A = tri_area(w[0], w[1], w[2]), A2 = tri_area(v[0], v[1], v[2]);
    const bool near = parents_touch(m.F, m.fparent[t], c2);
    double val[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int q = 0; q < 3; ++q) {
        const V3 x = tri_pt(c_r3, q, w[0], w[1], w[2]);
        const double wx = c_r3[q][3] * A;
        V3 m1 = {0, 0, 0};
        if (near) {
            YukAcc acc{kappa, false, true, 0.0, {0, 0, 0}, {0, 0, 0}};
            polar(x, v[0], v[1], v[2], nullptr, 0, false, acc);
            m1 = acc.mm1;
        } else {
            for (int q2 = 0; q2 < 7; ++q2) {
                const V3 ymx = tri_pt(c_r7, q2, v[0], v[1], v[2]) - x;
                const double R = nrm(ymx);
                const double g = c_r7[q2][3] * A2 * (1.0 + kappa * R) * exp(-kappa * R) / (4.0 * M_PI * R * R * R);
                m1 = m1 + g * ymx;
            }
        }
        for (int jj = 0; jj < 3; ++jj) {
            const V3 cr = (m.tsign[3 * c2 + jj] / (2.0 * A2)) * cross(x - v[jj], m1);
            for (int ii = 0; ii < 3; ++ii) val[ii][jj] += wx * dot((1.0 / (2.0 * A)) * (x - w[ii]), cr);
        }
    }
    for (int e = m.bc_ptr[t]; e < m.bc_ptr[t + 1]; ++e) {
        const double* ph = m.bc_phi + 3 * e;
        for (int jj = 0; jj < 3; ++jj) {
            const double vv = ph[0] * val[0][jj] + ph[1] * val[1][jj] + ph[2] * val[2][jj];
            if (vv != 0.0) atomicAdd(M + (int64_t)m.bc_fn[e] * m.ne + m.tedge[3 * c2 + jj], vv);
        }
    }
}

// G: one thread per fine triangle (degree-2 rule, exact for the quadratic integrand)
__global__ void k_gram(DevMesh m, double* __restrict__ G) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m.nf) return;
    const int c = m.fparent[t];
    const V3 w[3] = {mk(m.fV + 3 * m.fF[3 * t]), mk(m.fV + 3 * m.fF[3 * t + 1]), mk(m.fV + 3 * m.fF[3 * t + 2])};
    const V3 cv[3] = {mk(m.V + 3 * m.F[3 * c]), mk(m.V + 3 * m.F[3 * c + 1]), mk(m.V + 3 * m.F[3 * c + 2])};
    V3 nc = cross(cv[1] - cv[0], cv[2] - cv[0]);
    const double Ac = 0.5 * nrm(nc);
    nc = (1.0 / (2.0 * Ac)) * nc;
    const double A = tri_area(w[0], w[1], w[2]);
    for (int e = m.bc_ptr[t]; e < m.bc_ptr[t + 1]; ++e) {
        const double* ph = m.bc_phi + 3 * e;
        double acc[3] = {0, 0, 0};
        for (int q = 0; q < 3; ++q) {
            const V3 x = tri_pt(c_r3, q, w[0], w[1], w[2]);
            const V3 g = (1.0 / (2.0 * A)) * (ph[0] * (x - w[0]) + ph[1] * (x - w[1]) + ph[2] * (x - w[2]));
            const V3 ng = cross(nc, g);
            for (int j = 0; j < 3; ++j) {
                const V3 f = (m.tsign[3 * c + j] / (2.0 * Ac)) * (x - cv[j]);
                acc[j] += c_r3[q][3] * A * dot(ng, f);
            }
        }
        for (int j = 0; j < 3; ++j) atomicAdd(G + (int64_t)m.bc_fn[e] * m.ne + m.tedge[3 * c + j], acc[j]);
    }
}

static int* overflow_flag(cudaStream_t s) {
    static int* d = nullptr;
    if (!d) cudaMalloc(&d, sizeof(int));
    cudaMemsetAsync(d, 0, sizeof(int), s);
    return d;
}

static unsigned blocks(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

void launch_retarded_efie(const DevMesh& m, double dt, int K, double T0, double D, double* S, double* Phi,
                          int order, cudaStream_t s) {
    (void)D;
    cudaMemcpyToSymbolAsync(c_torder, &order, sizeof(int), 0, cudaMemcpyHostToDevice, s);
    int* of = overflow_flag(s);
    const int64_t n = (int64_t)m.nc * 7 * m.nc;
    k_retarded_efie<<<blocks(n, 128), 128, 0, s>>>(m, dt, K, T0, S, Phi, of);
}

void launch_retarded_mfie(const DevMesh& m, double dt, int K, double D, double* MM, int order, cudaStream_t s) {
    (void)D;
    cudaMemcpyToSymbolAsync(c_torder, &order, sizeof(int), 0, cudaMemcpyHostToDevice, s);
    int* of = overflow_flag(s);
    const int64_t n = (int64_t)m.nf * 3 * m.nc;
    k_retarded_mfie<<<blocks(n, 128), 128, 0, s>>>(m, dt, K, MM, of);
}

void launch_static(const DevMesh& m, double kappa, double* Zs, double* Psi, double* M, double* G, cudaStream_t s) {
    k_static_efie<<<blocks((int64_t)m.nf * m.nf, 128), 128, 0, s>>>(m, kappa, Zs, Psi);
    k_static_mfie<<<blocks((int64_t)m.nf * m.nc, 128), 128, 0, s>>>(m, kappa, M);
    k_gram<<<blocks(m.nf, 128), 128, 0, s>>>(m, G);
}

}  // namespace tdc
