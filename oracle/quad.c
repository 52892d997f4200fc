/*
 * oracle/quad.c -- plain, slow FP64 reference quadrature for the qHP TD-CFIE oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link or call this file;
 * only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg use it.
 *
 * It fills dense matrices of the space-time discretisation of Sec. II-C (RWG trial,
 * rotated RWG / rotated BC testing, Yukawa matrices) and of the Dirac-tested time
 * discretisation of Sec. IV-A.  Natural units: c = eta = 1.
 *
 * Every field is written with "local outward-flux fields" on a triangle t with
 * vertices w0, w1, w2 and area A:  L_{t,j}(r) = (r - w_j) / (2 A), the field with unit
 * outward flux through the edge opposite w_j.  A coarse RWG function (Sec. II-C,
 * Fig. 1) is +-L on its two triangles; a BC function is a combination of L's on the
 * fine triangles of the barycentric refinement (the coefficient table comes from
 * oracle/bc.py).
 *
 * Quadrature rule (the paper does not state one; both the oracle and the CUDA path
 * implement this same rule):
 *   outer: 7-point degree-5 rule on coarse triangles, 3-point degree-2 rule on fine ones.
 *   inner: polar decomposition about the projection p of the outer point onto the source
 *     plane (height d); one signed sub-triangle per edge; angular variable
 *     psi = asinh(lambda / h) along the edge (h = distance from p to the edge line),
 *     split where the circles R = R_b (the temporal breakpoints R_b = j*dt) cross the
 *     edge, and into pieces of width <= 1; radial variable u = asinh(rho / |d|)
 *     (rho itself when d = 0), split at the breakpoint radii and into pieces of width
 *     <= 1.  NANG Gauss-Legendre points per angular piece, NRAD per radial piece.
 *   retarded pairs (other than a triangle with itself) whose projection point p is well outside the
 *     source triangle (every vertex at least two longest edges from p): the same polar coordinates,
 *     but the angle runs over the triangle's own
 *     angular range seen from p, in two halves split at the middle vertex; in each half the
 *     angular variable is psi = asinh(tan(theta - theta_f)) along the nearer boundary edge
 *     (theta_f: its foot direction), split where breakpoint circles cross either boundary edge
 *     and into pieces of width <= 1; the radius runs from the near edge to the far edge (split at
 *     the breakpoint radii, u-variable pieces of width <= 1); no signed cancellation.
 *   static far pairs (parents share no vertex): product rules (3 x 3 fine-fine,
 *     3 x 7 fine-coarse).
 *   coplanar pairs (same coarse parent): the curl kernel vanishes identically
 *     (R-hat x f is normal, g is tangential) and is skipped.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define MAXG 32
#define MAXBRK 512
#define PI 3.14159265358979323846

static int NANG = 6, NRAD = 5;
static double PIECE = 1.0;
static double GA_X[MAXG], GA_W[MAXG], GR_X[MAXG], GR_W[MAXG];

/* Gauss-Legendre nodes/weights on [-1, 1] supplied by the caller (numpy.polynomial.legendre);
   piece: largest width of an angular (psi) or radial (u) sub-piece. */
void oq_set_rules(int na, const double* ax, const double* aw, int nr, const double* rx, const double* rw, double piece) {
    NANG = na; NRAD = nr; PIECE = piece;
    for (int i = 0; i < NANG; ++i) { GA_X[i] = ax[i]; GA_W[i] = aw[i]; }
    for (int i = 0; i < NRAD; ++i) { GR_X[i] = rx[i]; GR_W[i] = rw[i]; }
}

/* outer rules (barycentric coordinates + weights summing to 1) */
static const double R7_L[7][3] = {
    {1.0 / 3, 1.0 / 3, 1.0 / 3},
    {0.05971587178976982, 0.47014206410511511, 0.47014206410511511},
    {0.47014206410511511, 0.05971587178976982, 0.47014206410511511},
    {0.47014206410511511, 0.47014206410511511, 0.05971587178976982},
    {0.79742698535308731, 0.10128650732345634, 0.10128650732345634},
    {0.10128650732345634, 0.79742698535308731, 0.10128650732345634},
    {0.10128650732345634, 0.10128650732345634, 0.79742698535308731}};
static const double R7_W[7] = {0.225, 0.13239415278850619, 0.13239415278850619, 0.13239415278850619,
                               0.12593918054482714, 0.12593918054482714, 0.12593918054482714};
static const double R3_L[3][3] = {{2.0 / 3, 1.0 / 6, 1.0 / 6}, {1.0 / 6, 2.0 / 3, 1.0 / 6}, {1.0 / 6, 1.0 / 6, 2.0 / 3}};
static const double R3_W[3] = {1.0 / 3, 1.0 / 3, 1.0 / 3};

static inline void sub3(const double* a, const double* b, double* o) { o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2]; }
static inline double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static inline void cross3(const double* a, const double* b, double* o) {
    o[0] = a[1] * b[2] - a[2] * b[1]; o[1] = a[2] * b[0] - a[0] * b[2]; o[2] = a[0] * b[1] - a[1] * b[0];
}
static inline double norm3(const double* a) { return sqrt(dot3(a, a)); }

typedef void (*point_cb)(void* ctx, double R, double W, const double* ymx);
static int share_vertex(const int* F, int a, int b);


/* Integrate a function of y over the triangle (v0, v1, v2) for the outer point x:
   calls cb(ctx, R, W, y - x) at every inner node; the sum of W*G(y) approximates the
   integral.  brk: ascending breakpoint distances R_b (may be empty).  coplanar: the
   outer point lies in the source plane by construction (d := 0). */
static void polar_rule(const double* x, const double* v0, const double* v1, const double* v2,
                       const double* brk, int nbrk, int coplanar, point_cb cb, void* ctx) {
    double e1[3], e2[3], n[3], tmp[3];
    sub3(v1, v0, e1); sub3(v2, v0, e2); cross3(e1, e2, n);
    double nn = norm3(n);
    n[0] /= nn; n[1] /= nn; n[2] /= nn;
    sub3(x, v0, tmp);
    double d = coplanar ? 0.0 : dot3(tmp, n);
    double ad = fabs(d);
    double p[3] = {x[0] - d * n[0], x[1] - d * n[1], x[2] - d * n[2]};
    const double* V[3] = {v0, v1, v2};
    /* breakpoint radii in the plane */
    double rb[MAXBRK]; int nrb = 0;
    for (int b = 0; b < nbrk; ++b) if (brk[b] > ad) rb[nrb++] = sqrt(brk[b] * brk[b] - d * d);
    for (int s = 0; s < 3; ++s) {
        const double* a = V[s]; const double* b = V[(s + 1) % 3];
        double ab[3], pa[3], pb[3], cr[3];
        sub3(b, a, ab); double L = norm3(ab);
        double e[3] = {ab[0] / L, ab[1] / L, ab[2] / L};
        sub3(a, p, pa); sub3(b, p, pb); cross3(pa, pb, cr);
        double sig = dot3(cr, n);
        if (sig == 0.0) continue;
        sig = sig > 0 ? 1.0 : -1.0;
        double ap[3]; sub3(p, a, ap);
        double t = dot3(ap, e);
        double f[3] = {a[0] + t * e[0], a[1] + t * e[1], a[2] + t * e[2]};
        double nu[3]; sub3(f, p, nu);
        double h = norm3(nu);
        if (h <= 1e-14 * L) continue;
        nu[0] /= h; nu[1] /= h; nu[2] /= h;
        double la = -t, lb = L - t;               /* positions of a, b along e from the foot */
        double psa = asinh(la / h), psb = asinh(lb / h);
        /* angular split points */
        double sp[2 * MAXBRK + 2]; int nsp = 0;
        sp[nsp++] = psa;
        for (int q = 0; q < nrb; ++q) {
            if (rb[q] > h) {
                double c = acosh(rb[q] / h);
                if (-c > psa && -c < psb) sp[nsp++] = -c;
                if (c > psa && c < psb) sp[nsp++] = c;
            }
        }
        sp[nsp++] = psb;
        /* sort (insertion) */
        for (int i = 1; i < nsp; ++i) { double v = sp[i]; int j = i - 1; while (j >= 0 && sp[j] > v) { sp[j + 1] = sp[j]; --j; } sp[j + 1] = v; }
        for (int piece = 0; piece + 1 < nsp; ++piece) {
            double P0 = sp[piece], P1 = sp[piece + 1];
            if (P1 <= P0) continue;
            int nsub = (int)ceil((P1 - P0) / PIECE);
            if (nsub < 1) nsub = 1;
            double hw = (P1 - P0) / nsub;
            for (int sb = 0; sb < nsub; ++sb) {
                double q0 = P0 + sb * hw;
                for (int ga = 0; ga < NANG; ++ga) {
                    double psi = q0 + 0.5 * hw * (GA_X[ga] + 1.0);
                    double wpsi = 0.5 * hw * GA_W[ga];
                    double ch = cosh(psi), sh = sinh(psi);
                    double om[3] = {(nu[0] + sh * e[0]) / ch, (nu[1] + sh * e[1]) / ch, (nu[2] + sh * e[2]) / ch};
                    double rhoe = h * ch;
                    double ang = sig * wpsi / ch;
                    /* radial pieces */
                    double rp[MAXBRK + 2]; int nrp = 0;
                    rp[nrp++] = 0.0;
                    for (int q = 0; q < nrb; ++q) if (rb[q] > 0.0 && rb[q] < rhoe) rp[nrp++] = rb[q];
                    rp[nrp++] = rhoe;
                    for (int i = 1; i < nrp; ++i) { double v = rp[i]; int j = i - 1; while (j >= 0 && rp[j] > v) { rp[j + 1] = rp[j]; --j; } rp[j + 1] = v; }
                    for (int rpi = 0; rpi + 1 < nrp; ++rpi) {
                        double r0 = rp[rpi], r1 = rp[rpi + 1];
                        if (r1 <= r0) continue;
                        if (ad > 0.0) {
                            double u0 = asinh(r0 / ad), u1 = asinh(r1 / ad);
                            int ns = (int)ceil((u1 - u0) / PIECE);
                            if (ns < 1) ns = 1;
                            double uw = (u1 - u0) / ns;
                            for (int k = 0; k < ns; ++k) {
                                double ua = u0 + k * uw;
                                for (int gr = 0; gr < NRAD; ++gr) {
                                    double u = ua + 0.5 * uw * (GR_X[gr] + 1.0);
                                    double rho = ad * sinh(u), R = ad * cosh(u);
                                    double W = ang * 0.5 * uw * GR_W[gr] * rho * R;
                                    double ymx[3] = {rho * om[0] - d * n[0], rho * om[1] - d * n[1], rho * om[2] - d * n[2]};
                                    cb(ctx, R, W, ymx);
                                }
                            }
                        } else {
                            double rw = r1 - r0;
                            for (int gr = 0; gr < NRAD; ++gr) {
                                double rho = r0 + 0.5 * rw * (GR_X[gr] + 1.0);
                                double W = ang * 0.5 * rw * GR_W[gr] * rho;
                                double ymx[3] = {rho * om[0], rho * om[1], rho * om[2]};
                                cb(ctx, rho, W, ymx);
                            }
                        }
                    }
                }
            }
        }
    }
}


/* 2-D cross product */
static inline double cr2(double ax, double ay, double bx, double by) { return ax * by - ay * bx; }

/* Far-pair rule: integrate over the triangle only, in polar coordinates about p (projection of x),
   when p lies outside the triangle; otherwise the sub-triangle rule above (all signs positive). */
static void polar_far(const double* x, const double* v0, const double* v1, const double* v2,
                      const double* brk, int nbrk, point_cb cb, void* ctx) {
    double e1[3], e2[3], n[3], tmp[3];
    sub3(v1, v0, e1); sub3(v2, v0, e2); cross3(e1, e2, n);
    double nn = norm3(n);
    n[0] /= nn; n[1] /= nn; n[2] /= nn;
    sub3(x, v0, tmp);
    double d = dot3(tmp, n);
    double ad = fabs(d);
    double p[3] = {x[0] - d * n[0], x[1] - d * n[1], x[2] - d * n[2]};
    const double* V[3] = {v0, v1, v2};
    /* inside test: signed areas of (p, v_i, v_{i+1}) all >= 0 */
    int inside = 1;
    for (int i = 0; i < 3; ++i) {
        double a[3], b[3], c[3];
        sub3(V[i], p, a); sub3(V[(i + 1) % 3], p, b); cross3(a, b, c);
        if (dot3(c, n) < 0.0) inside = 0;
    }
    /* the far form only when p is well outside: every vertex at least two longest edges away */
    double lmax = 0.0, vmin = 1e300;
    for (int i = 0; i < 3; ++i) {
        double a[3], b[3];
        sub3(V[(i + 1) % 3], V[i], a);
        lmax = fmax(lmax, norm3(a));
        sub3(V[i], p, b);
        vmin = fmin(vmin, norm3(b));
    }
    if (inside || vmin < 2.0 * lmax) { polar_rule(x, v0, v1, v2, brk, nbrk, 0, cb, ctx); return; }
    /* in-plane frame: u toward the centroid, w = n x u */
    double g[3] = {(v0[0] + v1[0] + v2[0]) / 3.0 - p[0], (v0[1] + v1[1] + v2[1]) / 3.0 - p[1], (v0[2] + v1[2] + v2[2]) / 3.0 - p[2]};
    double gl = norm3(g);
    double u[3] = {g[0] / gl, g[1] / gl, g[2] / gl}, w[3];
    cross3(n, u, w);
    double X[3], Y[3], ph[3];
    for (int i = 0; i < 3; ++i) {
        double a[3];
        sub3(V[i], p, a);
        X[i] = dot3(a, u); Y[i] = dot3(a, w);
        ph[i] = atan2(Y[i], X[i]);
    }
    int o[3] = {0, 1, 2};
    for (int i = 1; i < 3; ++i) { int t = o[i], j = i - 1; while (j >= 0 && ph[o[j]] > ph[t]) { o[j + 1] = o[j]; --j; } o[j + 1] = t; }
    const int L = o[0], Mv = o[1], H = o[2];
    double rb[MAXBRK]; int nrb = 0;
    for (int b = 0; b < nbrk; ++b) if (brk[b] > ad) rb[nrb++] = sqrt(brk[b] * brk[b] - d * d);
    /* two angular halves: [phi_L, phi_M] bounded by edges LH and LM, [phi_M, phi_H] by LH and MH */
    for (int half = 0; half < 2; ++half) {
        const double P0 = half == 0 ? ph[L] : ph[Mv], P1 = half == 0 ? ph[Mv] : ph[H];
        if (!(P1 > P0)) continue;
        const int ea[2] = {L, half == 0 ? L : Mv}, eb[2] = {H, half == 0 ? Mv : H};
        /* near edge: the one the mid-angle ray meets first */
        double re_mid[2];
        {
            const double th = 0.5 * (P0 + P1), c = cos(th), sn = sin(th);
            for (int ei = 0; ei < 2; ++ei) {
                const double ax = X[ea[ei]], ay = Y[ea[ei]], bx = X[eb[ei]], by = Y[eb[ei]];
                re_mid[ei] = cr2(ax, ay, bx - ax, by - ay) / cr2(c, sn, bx - ax, by - ay);
            }
        }
        const int en = re_mid[0] < re_mid[1] ? 0 : 1;
        /* foot of the perpendicular from p on the near edge line: distance hn, angle thf */
        const double nax = X[ea[en]], nay = Y[ea[en]], nbx = X[eb[en]], nby = Y[eb[en]];
        const double ndx = nbx - nax, ndy = nby - nay, nl2 = ndx * ndx + ndy * ndy;
        const double tf = -(nax * ndx + nay * ndy) / nl2;
        const double fx = nax + tf * ndx, fy = nay + tf * ndy;
        const double hn = sqrt(fx * fx + fy * fy);
        if (!(hn > 0.0)) continue;
        const double thf = atan2(fy, fx);
        /* split angles: crossings of the breakpoint circles with both boundary edges */
        double sp[2 * 2 * MAXBRK + 2]; int nsp = 0;
        sp[nsp++] = P0;
        for (int ei = 0; ei < 2; ++ei) {
            const double ax = X[ea[ei]], ay = Y[ea[ei]], bx = X[eb[ei]], by = Y[eb[ei]];
            const double dx = bx - ax, dy = by - ay, dd = dx * dx + dy * dy;
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
        for (int i = 1; i < nsp; ++i) { double v = sp[i]; int j = i - 1; while (j >= 0 && sp[j] > v) { sp[j + 1] = sp[j]; --j; } sp[j + 1] = v; }
        /* angular variable psi = asinh(tan(theta - thf)) along the near edge; d theta = d psi / cosh psi */
        for (int piece = 0; piece + 1 < nsp; ++piece) {
            const double S0 = asinh(tan(sp[piece] - thf)), S1 = asinh(tan(sp[piece + 1] - thf));
            if (!(S1 > S0)) continue;
            int nsub = (int)ceil((S1 - S0) / PIECE);
            if (nsub < 1) nsub = 1;
            const double hw = (S1 - S0) / nsub;
            for (int sb = 0; sb < nsub; ++sb) {
                for (int ga = 0; ga < NANG; ++ga) {
                    const double psi = S0 + sb * hw + 0.5 * hw * (GA_X[ga] + 1.0);
                    const double wth = 0.5 * hw * GA_W[ga] / cosh(psi);
                    const double th = thf + atan(sinh(psi));
                    const double c = cos(th), sn = sin(th);
                    double re[2];
                    for (int ei = 0; ei < 2; ++ei) {
                        const double ax = X[ea[ei]], ay = Y[ea[ei]], bx = X[eb[ei]], by = Y[eb[ei]];
                        re[ei] = cr2(ax, ay, bx - ax, by - ay) / cr2(c, sn, bx - ax, by - ay);
                    }
                    const double r0 = re[en], r1 = re[1 - en];
                    double om[3] = {c * u[0] + sn * w[0], c * u[1] + sn * w[1], c * u[2] + sn * w[2]};
                    double rp[MAXBRK + 2]; int nrp = 0;
                    rp[nrp++] = r0;
                    for (int q = 0; q < nrb; ++q) if (rb[q] > r0 && rb[q] < r1) rp[nrp++] = rb[q];
                    rp[nrp++] = r1;
                    for (int i = 1; i < nrp; ++i) { double v = rp[i]; int j = i - 1; while (j >= 0 && rp[j] > v) { rp[j + 1] = rp[j]; --j; } rp[j + 1] = v; }
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
                                    const double uu = u0 + k * uw + 0.5 * uw * (GR_X[gr] + 1.0);
                                    const double rho = ad * sinh(uu), R = ad * cosh(uu);
                                    const double W = wth * 0.5 * uw * GR_W[gr] * rho * R;
                                    double ymx[3] = {rho * om[0] - d * n[0], rho * om[1] - d * n[1], rho * om[2] - d * n[2]};
                                    cb(ctx, R, W, ymx);
                                }
                        } else {
                            const double rw = a1 - a0;
                            for (int gr = 0; gr < NRAD; ++gr) {
                                const double rho = a0 + 0.5 * rw * (GR_X[gr] + 1.0);
                                double ymx[3] = {rho * om[0], rho * om[1], rho * om[2]};
                                cb(ctx, rho, wth * 0.5 * rw * GR_W[gr] * rho, ymx);
                            }
                        }
                    }
                }
            }
        }
    }
}

/* ---------------- temporal basis (Sec. IV-A) ----------------
 * Order 1 (the paper's pair): h0 the hat on [-dt, dt], q0 the C1 quadratic on [-dt, 2 dt].
 * Order 2 (the remark closing Sec. IV-B): h0 the shifted quadratic Lagrange interpolator, i.e.
 * on [(m-1) dt, m dt] the unknown is interpolated through t_m, t_{m-1}, t_{m-2}; with s = t/dt
 *   h0 = (s+1)(s+2)/2 on [-1, 0),  1 - s^2 on [0, 1),  (s-1)(s-2)/2 on [1, 2],
 * and q0 the function with q0' = (h0(t) - h0(t - dt))/dt that vanishes before -dt:
 *   q0(s) = H(s) - H(s - 1),  H(s) = int_{-1}^{s} h0 (dimensionless),
 * which is zero again after 3 dt because int h0 = 1. */
static int TORD = 1;
void oq_set_time_order(int p) { TORD = (p == 2) ? 2 : 1; }
int oq_time_order(void) { return TORD; }

static double H2(double s) {          /* int_{-1}^{s} of the order-2 h0 */
    if (s <= -1.0) return 0.0;
    if (s < 0.0) { double u = s + 1.0; return u * u * u / 6.0 + u * u / 4.0; }
    if (s < 1.0) return 5.0 / 12.0 + s - s * s * s / 3.0;
    if (s < 2.0) { double v = s - 1.0; return 13.0 / 12.0 + v * v * v / 6.0 - v * v / 4.0; }
    return 1.0;
}
static double h0(double t, double dt) {
    double s = t / dt;
    if (TORD == 2) {
        if (s >= -1.0 && s < 0.0) return 0.5 * (s + 1.0) * (s + 2.0);
        if (s >= 0.0 && s < 1.0) return 1.0 - s * s;
        if (s >= 1.0 && s <= 2.0) return 0.5 * (s - 1.0) * (s - 2.0);
        return 0.0;
    }
    if (t >= -dt && t < 0.0) return 1.0 + t / dt;
    if (t >= 0.0 && t <= dt) return 1.0 - t / dt;
    return 0.0;
}
static double h0dot(double t, double dt) {
    double s = t / dt;
    if (TORD == 2) {
        if (s > -1.0 && s < 0.0) return (s + 1.5) / dt;
        if (s > 0.0 && s < 1.0) return -2.0 * s / dt;
        if (s > 1.0 && s < 2.0) return (s - 1.5) / dt;
        return 0.0;
    }
    if (t > -dt && t < 0.0) return 1.0 / dt;
    if (t > 0.0 && t < dt) return -1.0 / dt;
    return 0.0;
}
static double q0(double t, double dt) {
    double s = t / dt;
    if (TORD == 2) return H2(s) - H2(s - 1.0);
    if (t >= -dt && t < 0.0) return 0.5 * (s + 1.0) * (s + 1.0);
    if (t >= 0.0 && t < dt) return 0.5 - s * s + s;
    if (t >= dt && t <= 2.0 * dt) return 0.5 * (s - 2.0) * (s - 2.0);
    return 0.0;
}

/* exported for the tests of the time basis */
double oq_h0(double t, double dt) { return h0(t, dt); }
double oq_h0dot(double t, double dt) { return h0dot(t, dt); }
double oq_q0(double t, double dt) { return q0(t, dt); }

/* ---------------- generic test hook: integrate moments of F over a triangle ---------------- */
typedef struct { int kind; double p1, p2; double m0; double m1[3]; } test_ctx;
static double h0(double t, double dt);
static double h0dot(double t, double dt);
static double q0(double t, double dt);
static void test_cb(void* c, double R, double W, const double* ymx) {
    test_ctx* t = (test_ctx*)c;
    double F = 0.0;
    if (t->kind == 0) F = 1.0;                      /* area / centroid */
    else if (t->kind == 1) F = 1.0 / R;             /* single-layer potential */
    else if (t->kind == 2) F = exp(-t->p1 * R) / R;  /* Yukawa, p1 = kappa */
    else if (t->kind == 3) F = 1.0 / (R * R * R);   /* double-layer type */
    else if (t->kind == 4) F = q0(t->p1 - R, t->p2) / R;       /* p1 = k dt, p2 = dt */
    else if (t->kind == 5) F = h0dot(t->p1 - R, t->p2) / R;
    else if (t->kind == 6) F = h0(t->p1 - R, t->p2) / (R * R * R);
    t->m0 += W * F;
    for (int i = 0; i < 3; ++i) t->m1[i] += W * F * ymx[i];
}
/* out: m0, m1[3] (moment about x).  coplanar: 0 general, 1 coplanar (d = 0), 2 far-pair rule.
   kind 0: 1, 1: 1/R, 2: exp(-p1 R)/R, 3: 1/R^3,
   4: q0(p1 - R)/R, 5: h0dot(p1 - R)/R, 6: h0(p1 - R)/R^3 (p2 = dt). */
void oq_triangle_moments(const double* x, const double* v0, const double* v1, const double* v2,
                         const double* brk, int nbrk, int coplanar, int kind, double p1, double p2, double* out) {
    test_ctx t = {kind, p1, p2, 0.0, {0, 0, 0}};
    if (coplanar == 2) polar_far(x, v0, v1, v2, brk, nbrk, test_cb, &t);   /* far-pair rule */
    else polar_rule(x, v0, v1, v2, brk, nbrk, coplanar, test_cb, &t);
    out[0] = t.m0; out[1] = t.m1[0]; out[2] = t.m1[1]; out[3] = t.m1[2];
}

/* ---------------- retarded accumulation ---------------- */
typedef struct {
    int K; double dt; double T0;
    double* s0; double* s1;     /* K, K*3 : F_S = -h0dot/(4 pi R) */
    double* p0;                 /* K     : F_Phi = -T0 q0/(4 pi R) */
    double* m0; double* m1;     /* K, K*3 : F_M = (h0/R + h0dot)/(4 pi R^2) */
    int want_sp, want_m;
} ret_ctx;

static void ret_cb(void* c, double R, double W, const double* ymx) {
    ret_ctx* r = (ret_ctx*)c;
    for (int k = 0; k < r->K; ++k) {
        double tau = k * r->dt - R;
        if (tau <= -r->dt || tau >= (TORD + 1) * r->dt) continue;     /* support of q0 */
        double hd = h0dot(tau, r->dt), hv = h0(tau, r->dt), qv = q0(tau, r->dt);
        if (r->want_sp) {
            double fs = -hd / (4.0 * PI * R);
            r->s0[k] += W * fs;
            for (int i = 0; i < 3; ++i) r->s1[3 * k + i] += W * fs * ymx[i];
            r->p0[k] += W * (-r->T0 * qv / (4.0 * PI * R));
        }
        if (r->want_m) {
            double fm = (hv / R + hd) / (4.0 * PI * R * R);
            r->m0[k] += W * fm;
            for (int i = 0; i < 3; ++i) r->m1[3 * k + i] += W * fm * ymx[i];
        }
    }
}

static double tri_area(const double* a, const double* b, const double* c, double* nrm) {
    double e1[3], e2[3], n[3];
    sub3(b, a, e1); sub3(c, a, e2); cross3(e1, e2, n);
    double l = norm3(n);
    if (nrm) { nrm[0] = n[0] / l; nrm[1] = n[1] / l; nrm[2] = n[2] / l; }
    return 0.5 * l;
}

static int breakpoints(double dt, double Rmax, double* brk) {
    int nb = 0;
    for (int j = 1; j * dt <= Rmax + dt && nb < MAXBRK; ++j) brk[nb++] = j * dt;
    return nb;
}

/*
 * S_k[m,n]  = -int int f_m(x).f_n(y) h0dot(k dt - R)/(4 pi R)            (EFIE vector potential)
 * Phi_k[c,c'] = -T0/(A_c A_c') int_c int_c' q0(k dt - R)/(4 pi R)        (EFIE scalar potential)
 * Coarse tables: F (nc x 3 vertex ids, CCW outward), tedge (nc x 3: edge of the local edge
 * opposite vertex j), tsign (nc x 3: +1 if the triangle is c+ of that edge, else -1).
 * Output layout: S[k][m][n] (K x ne x ne), Phi[k][c][c'] (K x nc x nc), row-major, zeroed by caller.
 */
void oq_retarded_efie(const double* Vx, int nc, const int* F, int ne, const int* tedge, const double* tsign,
                      double dt, int K, double T0, double Rmax, double* S, double* Phi) {
    double brk[MAXBRK];
    int nb = breakpoints(dt, Rmax, brk);
#pragma omp parallel for schedule(dynamic, 1)
    for (int c = 0; c < nc; ++c) {
        const double* w[3] = {Vx + 3 * F[3 * c], Vx + 3 * F[3 * c + 1], Vx + 3 * F[3 * c + 2]};
        double A = tri_area(w[0], w[1], w[2], NULL);
        double* rowS = (double*)calloc((size_t)3 * K * ne, sizeof(double));
        double* rowP = (double*)calloc((size_t)K * nc, sizeof(double));
        double* s0 = (double*)malloc(sizeof(double) * K);
        double* s1 = (double*)malloc(sizeof(double) * 3 * K);
        double* p0 = (double*)malloc(sizeof(double) * K);
        for (int q = 0; q < 7; ++q) {
            double x[3];
            for (int i = 0; i < 3; ++i) x[i] = R7_L[q][0] * w[0][i] + R7_L[q][1] * w[1][i] + R7_L[q][2] * w[2][i];
            double wx = R7_W[q] * A;
            for (int c2 = 0; c2 < nc; ++c2) {
                const double* v[3] = {Vx + 3 * F[3 * c2], Vx + 3 * F[3 * c2 + 1], Vx + 3 * F[3 * c2 + 2]};
                double A2 = tri_area(v[0], v[1], v[2], NULL);
                memset(s0, 0, sizeof(double) * K); memset(s1, 0, sizeof(double) * 3 * K); memset(p0, 0, sizeof(double) * K);
                ret_ctx r = {K, dt, T0, s0, s1, p0, NULL, NULL, 1, 0};
                if (c2 == c) polar_rule(x, v[0], v[1], v[2], brk, nb, 1, ret_cb, &r);
                else polar_far(x, v[0], v[1], v[2], brk, nb, ret_cb, &r);
                for (int k = 0; k < K; ++k) {
                    rowP[(size_t)k * nc + c2] += wx * p0[k] / (A * A2);
                    if (s0[k] == 0.0 && s1[3 * k] == 0.0 && s1[3 * k + 1] == 0.0 && s1[3 * k + 2] == 0.0) continue;
                    for (int i = 0; i < 3; ++i) {
                        double Lx[3];
                        for (int a = 0; a < 3; ++a) Lx[a] = tsign[3 * c + i] * (x[a] - w[i][a]) / (2.0 * A);
                        for (int j = 0; j < 3; ++j) {
                            /* int L_{c2,j}(y) F dy = (m1 + (x - v_j) m0) / (2 A2) */
                            double Iy[3];
                            for (int a = 0; a < 3; ++a) Iy[a] = tsign[3 * c2 + j] * (s1[3 * k + a] + (x[a] - v[j][a]) * s0[k]) / (2.0 * A2);
                            rowS[((size_t)i * K + k) * ne + tedge[3 * c2 + j]] += wx * dot3(Lx, Iy);
                        }
                    }
                }
            }
        }
#pragma omp critical
        {
            for (int i = 0; i < 3; ++i) {
                int m = tedge[3 * c + i];
                for (int k = 0; k < K; ++k)
                    for (int n = 0; n < ne; ++n) S[((size_t)k * ne + m) * ne + n] += rowS[((size_t)i * K + k) * ne + n];
            }
            for (int k = 0; k < K; ++k)
                for (int c2 = 0; c2 < nc; ++c2) Phi[((size_t)k * nc + c) * nc + c2] += rowP[(size_t)k * nc + c2];
        }
        free(rowS); free(rowP); free(s0); free(s1); free(p0);
    }
}

/*
 * MM_k[m,n] = int int g_m(x).[R-hat x f_n(y)] (h0(k dt - R)/(4 pi R^2) + h0dot(k dt - R)/(4 pi R))
 * BC tables (fine mesh): fV (fine vertices), fF (nf x 3), fparent (nf), and a CSR over fine
 * triangles: bc_ptr (nf+1), bc_fn (BC function index), bc_phi (3 outward fluxes per entry).
 * Output MM[k][m][n] (K x ne x ne), zeroed by caller.
 */
void oq_retarded_mfie(const double* Vx, int nc, const int* F, int ne, const int* tedge, const double* tsign,
                      const double* fV, int nf, const int* fF, const int* fparent,
                      const int* bc_ptr, const int* bc_fn, const double* bc_phi,
                      double dt, int K, double Rmax, double* MM) {
    double brk[MAXBRK];
    int nb = breakpoints(dt, Rmax, brk);
#pragma omp parallel for schedule(dynamic, 1)
    for (int t = 0; t < nf; ++t) {
        const double* w[3] = {fV + 3 * fF[3 * t], fV + 3 * fF[3 * t + 1], fV + 3 * fF[3 * t + 2]};
        double A = tri_area(w[0], w[1], w[2], NULL);
        /* local block: 3 outer local fields x K x ne */
        double* blk = (double*)calloc((size_t)3 * K * ne, sizeof(double));
        double* m0 = (double*)malloc(sizeof(double) * K);
        double* m1 = (double*)malloc(sizeof(double) * 3 * K);
        for (int q = 0; q < 3; ++q) {
            double x[3];
            for (int i = 0; i < 3; ++i) x[i] = R3_L[q][0] * w[0][i] + R3_L[q][1] * w[1][i] + R3_L[q][2] * w[2][i];
            double wx = R3_W[q] * A;
            for (int c2 = 0; c2 < nc; ++c2) {
                if (c2 == fparent[t]) continue;   /* coplanar: curl kernel vanishes */
                const double* v[3] = {Vx + 3 * F[3 * c2], Vx + 3 * F[3 * c2 + 1], Vx + 3 * F[3 * c2 + 2]};
                double A2 = tri_area(v[0], v[1], v[2], NULL);
                memset(m0, 0, sizeof(double) * K); memset(m1, 0, sizeof(double) * 3 * K);
                ret_ctx r = {K, dt, 0.0, NULL, NULL, NULL, m0, m1, 0, 1};
                polar_far(x, v[0], v[1], v[2], brk, nb, ret_cb, &r);
                for (int k = 0; k < K; ++k) {
                    if (m0[k] == 0.0 && m1[3 * k] == 0.0 && m1[3 * k + 1] == 0.0 && m1[3 * k + 2] == 0.0) continue;
                    for (int j = 0; j < 3; ++j) {
                        /* int [R-hat x L_{c2,j}(y)] F dy = (x - v_j) x m1 / (2 A2) */
                        double xv[3], cr[3];
                        sub3(x, v[j], xv);
                        cross3(xv, m1 + 3 * k, cr);
                        double s = tsign[3 * c2 + j] / (2.0 * A2);
                        for (int i = 0; i < 3; ++i) {
                            double Lx[3];
                            for (int a = 0; a < 3; ++a) Lx[a] = (x[a] - w[i][a]) / (2.0 * A);
                            blk[((size_t)i * K + k) * ne + tedge[3 * c2 + j]] += wx * s * dot3(Lx, cr);
                        }
                    }
                }
            }
        }
#pragma omp critical
        {
            for (int e = bc_ptr[t]; e < bc_ptr[t + 1]; ++e) {
                int m = bc_fn[e];
                for (int i = 0; i < 3; ++i) {
                    double ph = bc_phi[3 * e + i];
                    if (ph == 0.0) continue;
                    for (int k = 0; k < K; ++k)
                        for (int n = 0; n < ne; ++n) MM[((size_t)k * ne + m) * ne + n] += ph * blk[((size_t)i * K + k) * ne + n];
                }
            }
        }
        free(blk); free(m0); free(m1);
    }
}

/* ---------------- static (Yukawa) matrices ---------------- */
typedef struct { double kappa; double z0; double z1[3]; double mm0; double mm1[3]; int want_z, want_m; } sta_ctx;
static void sta_cb(void* c, double R, double W, const double* ymx) {
    sta_ctx* s = (sta_ctx*)c;
    double ek = exp(-s->kappa * R);
    if (s->want_z) {
        double g = ek / (4.0 * PI * R);
        s->z0 += W * g;
        for (int i = 0; i < 3; ++i) s->z1[i] += W * g * ymx[i];
    }
    if (s->want_m) {
        double g = (1.0 + s->kappa * R) * ek / (4.0 * PI * R * R * R);
        s->mm0 += W * g;
        for (int i = 0; i < 3; ++i) s->mm1[i] += W * g * ymx[i];
    }
}

static int share_vertex(const int* F, int a, int b) {
    for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) if (F[3 * a + i] == F[3 * b + j]) return 1;
    return 0;
}

/*
 * Zs[m,n]  = -kappa int int g_m(x).g_n(y) exp(-kappa R)/(4 pi R)
 * Psi[v,v'] = -(1/kappa) int int rho_v(x) rho_v'(y) exp(-kappa R)/(4 pi R),
 *             rho_v = 1/(2 N_v A_t) on each fine triangle t of the dual cell of v
 * fvert (nf): the coarse vertex of each fine triangle; nval (nv): coarse valence N_v.
 */
void oq_static_efie(const int* F, const double* fV, int nf, const int* fF, const int* fparent, const int* fvert,
                    const int* nval, int nv, const int* bc_ptr, const int* bc_fn, const double* bc_phi, int ne,
                    double kappa, double* Zs, double* Psi) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int t = 0; t < nf; ++t) {
        const double* w[3] = {fV + 3 * fF[3 * t], fV + 3 * fF[3 * t + 1], fV + 3 * fF[3 * t + 2]};
        double A = tri_area(w[0], w[1], w[2], NULL);
        /* I[i][t2][j] local dot integrals and scalar integral per t2 */
        double* Id = (double*)calloc((size_t)9 * nf, sizeof(double));
        double* Is = (double*)calloc((size_t)nf, sizeof(double));
        for (int t2 = 0; t2 < nf; ++t2) {
            const double* v[3] = {fV + 3 * fF[3 * t2], fV + 3 * fF[3 * t2 + 1], fV + 3 * fF[3 * t2 + 2]};
            double A2 = tri_area(v[0], v[1], v[2], NULL);
            int near = share_vertex(F, fparent[t], fparent[t2]);
            for (int q = 0; q < 3; ++q) {
                double x[3];
                for (int i = 0; i < 3; ++i) x[i] = R3_L[q][0] * w[0][i] + R3_L[q][1] * w[1][i] + R3_L[q][2] * w[2][i];
                double wx = R3_W[q] * A;
                double z0 = 0.0, z1[3] = {0, 0, 0};
                if (near) {
                    sta_ctx s = {kappa, 0.0, {0, 0, 0}, 0.0, {0, 0, 0}, 1, 0};
                    polar_rule(x, v[0], v[1], v[2], NULL, 0, fparent[t] == fparent[t2], sta_cb, &s);
                    z0 = s.z0; z1[0] = s.z1[0]; z1[1] = s.z1[1]; z1[2] = s.z1[2];
                } else {
                    for (int q2 = 0; q2 < 3; ++q2) {
                        double y[3], ymx[3];
                        for (int i = 0; i < 3; ++i) y[i] = R3_L[q2][0] * v[0][i] + R3_L[q2][1] * v[1][i] + R3_L[q2][2] * v[2][i];
                        sub3(y, x, ymx);
                        double R = norm3(ymx);
                        double g = R3_W[q2] * A2 * exp(-kappa * R) / (4.0 * PI * R);
                        z0 += g;
                        for (int i = 0; i < 3; ++i) z1[i] += g * ymx[i];
                    }
                }
                Is[t2] += wx * z0;
                for (int i = 0; i < 3; ++i) {
                    double Lx[3];
                    for (int a = 0; a < 3; ++a) Lx[a] = (x[a] - w[i][a]) / (2.0 * A);
                    for (int j = 0; j < 3; ++j) {
                        double Iy[3];
                        for (int a = 0; a < 3; ++a) Iy[a] = (z1[a] + (x[a] - v[j][a]) * z0) / (2.0 * A2);
                        Id[(size_t)(i * nf + t2) * 3 + j] += wx * dot3(Lx, Iy);
                    }
                }
            }
        }
#pragma omp critical
        {
            double rv = 1.0 / (2.0 * nval[fvert[t]] * A);
            for (int t2 = 0; t2 < nf; ++t2) {
                const double* v[3] = {fV + 3 * fF[3 * t2], fV + 3 * fF[3 * t2 + 1], fV + 3 * fF[3 * t2 + 2]};
                double A2 = tri_area(v[0], v[1], v[2], NULL);
                double rv2 = 1.0 / (2.0 * nval[fvert[t2]] * A2);
                Psi[(size_t)fvert[t] * nv + fvert[t2]] += -(1.0 / kappa) * rv * rv2 * Is[t2];
                for (int e1 = bc_ptr[t]; e1 < bc_ptr[t + 1]; ++e1)
                    for (int e2 = bc_ptr[t2]; e2 < bc_ptr[t2 + 1]; ++e2) {
                        double acc = 0.0;
                        for (int i = 0; i < 3; ++i)
                            for (int j = 0; j < 3; ++j)
                                acc += bc_phi[3 * e1 + i] * bc_phi[3 * e2 + j] * Id[(size_t)(i * nf + t2) * 3 + j];
                        Zs[(size_t)bc_fn[e1] * ne + bc_fn[e2]] += -kappa * acc;
                    }
            }
        }
        free(Id); free(Is);
    }
}

/* M[m,n] = int int g_m(x).[R-hat x f_n(y)] (1 + kappa R) exp(-kappa R)/(4 pi R^2) */
void oq_static_mfie(const double* Vx, int nc, const int* F, int ne, const int* tedge, const double* tsign,
                    const double* fV, int nf, const int* fF, const int* fparent,
                    const int* bc_ptr, const int* bc_fn, const double* bc_phi, double kappa, double* M) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int t = 0; t < nf; ++t) {
        const double* w[3] = {fV + 3 * fF[3 * t], fV + 3 * fF[3 * t + 1], fV + 3 * fF[3 * t + 2]};
        double A = tri_area(w[0], w[1], w[2], NULL);
        double* blk = (double*)calloc((size_t)3 * ne, sizeof(double));
        for (int c2 = 0; c2 < nc; ++c2) {
            if (c2 == fparent[t]) continue;
            const double* v[3] = {Vx + 3 * F[3 * c2], Vx + 3 * F[3 * c2 + 1], Vx + 3 * F[3 * c2 + 2]};
            double A2 = tri_area(v[0], v[1], v[2], NULL);
            int near = share_vertex(F, fparent[t], c2);
            for (int q = 0; q < 3; ++q) {
                double x[3];
                for (int i = 0; i < 3; ++i) x[i] = R3_L[q][0] * w[0][i] + R3_L[q][1] * w[1][i] + R3_L[q][2] * w[2][i];
                double wx = R3_W[q] * A;
                double m1[3] = {0, 0, 0};
                if (near) {
                    sta_ctx s = {kappa, 0.0, {0, 0, 0}, 0.0, {0, 0, 0}, 0, 1};
                    polar_rule(x, v[0], v[1], v[2], NULL, 0, 0, sta_cb, &s);
                    m1[0] = s.mm1[0]; m1[1] = s.mm1[1]; m1[2] = s.mm1[2];
                } else {
                    for (int q2 = 0; q2 < 7; ++q2) {
                        double y[3], ymx[3];
                        for (int i = 0; i < 3; ++i) y[i] = R7_L[q2][0] * v[0][i] + R7_L[q2][1] * v[1][i] + R7_L[q2][2] * v[2][i];
                        sub3(y, x, ymx);
                        double R = norm3(ymx);
                        double g = R7_W[q2] * A2 * (1.0 + kappa * R) * exp(-kappa * R) / (4.0 * PI * R * R * R);
                        for (int i = 0; i < 3; ++i) m1[i] += g * ymx[i];
                    }
                }
                for (int j = 0; j < 3; ++j) {
                    double xv[3], cr[3];
                    sub3(x, v[j], xv);
                    cross3(xv, m1, cr);
                    double s = tsign[3 * c2 + j] / (2.0 * A2);
                    for (int i = 0; i < 3; ++i) {
                        double Lx[3];
                        for (int a = 0; a < 3; ++a) Lx[a] = (x[a] - w[i][a]) / (2.0 * A);
                        blk[(size_t)i * ne + tedge[3 * c2 + j]] += wx * s * dot3(Lx, cr);
                    }
                }
            }
        }
#pragma omp critical
        {
            for (int e = bc_ptr[t]; e < bc_ptr[t + 1]; ++e)
                for (int i = 0; i < 3; ++i) {
                    double ph = bc_phi[3 * e + i];
                    if (ph == 0.0) continue;
                    for (int n = 0; n < ne; ++n) M[(size_t)bc_fn[e] * ne + n] += ph * blk[(size_t)i * ne + n];
                }
        }
        free(blk);
    }
}
