// Host-side mesh tables: validation, edge table, incidence (Sec. II-D), barycentric refinement
// and the Buffa-Christiansen coefficient table (Sec. II-C, Fig. 2).
//
// Edge orientation: v- = smaller vertex index, v+ = larger; c+ is the triangle whose
// counter-clockwise cycle runs v- -> v+ (then Sigma^T Lambda = 0 and RWG loops are div-free).
//
// BC function g_n (unit-flux fine-RWG form): unit flux leaves the dual cell of v+ across the
// dual edge of e_n (1/2 through each of the two fine edges midpoint-barycentre) into the dual
// cell of v-; inside a cell with N coarse triangles the flux through the radial fine edges
// changes by 1/(2N) per fine triangle, with zero flux through the coarse half edge of e_n, so
// every fine triangle of the source (sink) cell carries charge +1/(2N) (-1/(2N)).
#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <numeric>
#include <set>
#include <tuple>

#include "internal.h"

namespace tdc {

namespace {
struct DSU {
    std::vector<int> p;
    explicit DSU(int n) : p(n) { std::iota(p.begin(), p.end(), 0); }
    int find(int x) { while (p[x] != x) { p[x] = p[p[x]]; x = p[x]; } return x; }
    void join(int a, int b) { a = find(a); b = find(b); if (a != b) p[a] = b; }
};
}  // namespace

std::string build_mesh(const double* V, int64_t nv64, const int32_t* F, int64_t nc64, Mesh& m) {
    if (nv64 < 4 || nc64 < 4 || nv64 > (1 << 26) || nc64 > (1 << 26)) return "mesh size out of range";
    const int nv = (int)nv64, nc = (int)nc64;
    m.nv = nv; m.nc = nc;
    m.V.assign(V, V + 3 * (size_t)nv);
    m.F.assign(F, F + 3 * (size_t)nc);
    for (int i = 0; i < 3 * nc; ++i)
        if (m.F[i] < 0 || m.F[i] >= nv) return "triangle references a vertex out of range";
    for (int c = 0; c < nc; ++c) {
        const int a = m.F[3 * c], b = m.F[3 * c + 1], d = m.F[3 * c + 2];
        if (a == b || b == d || a == d) return "degenerate triangle (repeated vertex)";
    }
    for (double x : m.V) if (!std::isfinite(x)) return "non-finite vertex coordinate";
    // directed half-edges: (a, b) -> triangle whose CCW cycle runs a -> b
    std::map<std::pair<int, int>, int> half;
    for (int c = 0; c < nc; ++c)
        for (int j = 0; j < 3; ++j) {
            const int a = m.F[3 * c + (j + 1) % 3], b = m.F[3 * c + (j + 2) % 3];
            if (!half.emplace(std::make_pair(a, b), c).second)
                return "edge used twice in the same direction (non-manifold or inconsistent orientation)";
        }
    // undirected edges, lexicographic
    std::vector<std::pair<int, int>> und;
    und.reserve(half.size() / 2 + 1);
    for (auto& kv : half) {
        const int a = kv.first.first, b = kv.first.second;
        if (!half.count({b, a})) return "open edge (surface not closed)";
        if (a < b) und.emplace_back(a, b);
    }
    std::sort(und.begin(), und.end());
    const int ne = (int)und.size();
    m.ne = ne;
    m.E.resize(2 * (size_t)ne);
    m.cplus.resize(ne); m.cminus.resize(ne);
    std::map<std::pair<int, int>, int> eid;
    for (int i = 0; i < ne; ++i) {
        m.E[2 * i] = und[i].first; m.E[2 * i + 1] = und[i].second;
        m.cplus[i] = half[{und[i].first, und[i].second}];
        m.cminus[i] = half[{und[i].second, und[i].first}];
        eid[und[i]] = i;
    }
    m.tedge.resize(3 * (size_t)nc); m.tsign.resize(3 * (size_t)nc);
    for (int c = 0; c < nc; ++c)
        for (int j = 0; j < 3; ++j) {
            const int a = m.F[3 * c + (j + 1) % 3], b = m.F[3 * c + (j + 2) % 3];
            const int e = eid[{std::min(a, b), std::max(a, b)}];
            m.tedge[3 * c + j] = e;
            m.tsign[3 * c + j] = (a < b) ? 1.0 : -1.0;
        }
    DSU dsu(nc);
    for (int e = 0; e < ne; ++e) dsu.join(m.cplus[e], m.cminus[e]);
    for (int c = 1; c < nc; ++c) if (dsu.find(c) != dsu.find(0)) return "surface is not connected";
    m.valence.assign(nv, 0);
    for (int i = 0; i < 3 * nc; ++i) m.valence[m.F[i]]++;
    for (int v = 0; v < nv; ++v) if (m.valence[v] < 3) return "vertex with fewer than 3 triangles (unused or pinched)";
    const int chi = nv - ne + nc;
    if (chi > 2 || (chi & 1)) return "Euler characteristic of a non-orientable or non-closed surface";
    m.genus = (2 - chi) / 2;
    double D = 0.0;
    for (int i = 0; i < nv; ++i)
        for (int j = i + 1; j < nv; ++j) {
            const double dx = m.V[3 * i] - m.V[3 * j], dy = m.V[3 * i + 1] - m.V[3 * j + 1], dz = m.V[3 * i + 2] - m.V[3 * j + 2];
            D = std::max(D, dx * dx + dy * dy + dz * dz);
        }
    m.D = std::sqrt(D);

    // ---------------- barycentric refinement
    const int nfv = nv + ne + nc;
    m.fV.resize(3 * (size_t)nfv);
    for (int i = 0; i < 3 * nv; ++i) m.fV[i] = m.V[i];
    for (int e = 0; e < ne; ++e)
        for (int k = 0; k < 3; ++k)
            m.fV[3 * (nv + e) + k] = 0.5 * (m.V[3 * m.E[2 * e] + k] + m.V[3 * m.E[2 * e + 1] + k]);
    for (int c = 0; c < nc; ++c)
        for (int k = 0; k < 3; ++k)
            m.fV[3 * (nv + ne + c) + k] =
                (m.V[3 * m.F[3 * c] + k] + m.V[3 * m.F[3 * c + 1] + k] + m.V[3 * m.F[3 * c + 2] + k]) / 3.0;
    m.nf = 6 * nc;
    m.fF.resize(3 * (size_t)m.nf); m.fparent.resize(m.nf); m.fvert.resize(m.nf);
    // fine triangle of coarse c at local vertex j: slot 0 borders the edge to the next vertex,
    // slot 1 the edge to the previous vertex
    auto fidx = [](int c, int j, int slot) { return 6 * c + 2 * j + slot; };
    for (int c = 0; c < nc; ++c) {
        const int bary = nv + ne + c;
        for (int j = 0; j < 3; ++j) {
            const int u = m.F[3 * c + j];
            const int enext = m.tedge[3 * c + (j + 2) % 3];   // edge {u, F[j+1]}
            const int eprev = m.tedge[3 * c + (j + 1) % 3];   // edge {F[j+2], u}
            int t0 = fidx(c, j, 0), t1 = fidx(c, j, 1);
            m.fF[3 * t0] = u; m.fF[3 * t0 + 1] = nv + enext; m.fF[3 * t0 + 2] = bary;
            m.fF[3 * t1] = u; m.fF[3 * t1 + 1] = bary; m.fF[3 * t1 + 2] = nv + eprev;
            m.fparent[t0] = m.fparent[t1] = c;
            m.fvert[t0] = m.fvert[t1] = u;
        }
    }
    // locate, for coarse c and its vertex u, the fine triangle bordering coarse edge e
    auto fine_at = [&](int c, int u, int e) -> int {
        for (int j = 0; j < 3; ++j)
            if (m.F[3 * c + j] == u) {
                if (m.tedge[3 * c + (j + 2) % 3] == e) return fidx(c, j, 0);
                if (m.tedge[3 * c + (j + 1) % 3] == e) return fidx(c, j, 1);
            }
        return -1;
    };
    // local index (0..2) of the fine edge shared by fine triangles a and b, seen from a
    auto shared_local = [&](int a, int b) -> int {
        for (int j = 0; j < 3; ++j) {
            const int p = m.fF[3 * a + (j + 1) % 3], q = m.fF[3 * a + (j + 2) % 3];
            int hit = 0;
            for (int k = 0; k < 3; ++k) hit += (m.fF[3 * b + k] == p) + (m.fF[3 * b + k] == q);
            if (hit == 2) return j;
        }
        return -1;
    };
    std::map<std::pair<int, int>, std::array<double, 3>> flux;   // (fine tri, fn) -> outward fluxes
    auto add_flux = [&](int n, int from, int to, double phi) -> bool {
        if (phi == 0.0) return true;
        const int ja = shared_local(from, to), jb = shared_local(to, from);
        if (ja < 0 || jb < 0) return false;
        flux[{from, n}][ja] += phi;
        flux[{to, n}][jb] -= phi;
        return true;
    };
    // fan of fine triangles around coarse vertex v, starting in coarse triangle c0 next to the
    // half edge of coarse edge e0 and moving away from it
    auto fan = [&](int v, int c0, int e0, std::vector<int>& out) -> bool {
        out.clear();
        int c = c0, e = e0;
        for (int guard = 0; guard < 4 * nc + 8; ++guard) {
            out.push_back(fine_at(c, v, e));
            int other = -1;
            for (int j = 0; j < 3; ++j)
                if (m.F[3 * c + j] == v) {
                    const int a = m.tedge[3 * c + (j + 1) % 3], b = m.tedge[3 * c + (j + 2) % 3];
                    other = (a == e) ? b : a;
                }
            out.push_back(fine_at(c, v, other));
            c = (m.cplus[other] == c) ? m.cminus[other] : m.cplus[other];
            e = other;
            if (e == e0) return (int)out.size() == 2 * m.valence[v];
        }
        return false;
    };
    std::vector<int> cyc;
    for (int n = 0; n < ne; ++n) {
        const int vm = m.E[2 * n], vp = m.E[2 * n + 1];
        const int cp = m.cplus[n], cm = m.cminus[n];
        for (int c : {cp, cm})
            if (!add_flux(n, fine_at(c, vp, n), fine_at(c, vm, n), 0.5)) return "BC construction failed (dual edge)";
        if (!fan(vm, cp, n, cyc)) return "non-manifold vertex fan";
        int N = (int)cyc.size() / 2;
        for (int i = 1; i < 2 * N; ++i)
            if (!add_flux(n, cyc[i - 1], cyc[i], 0.5 - i / (2.0 * N))) return "BC construction failed (sink fan)";
        if (!fan(vp, cp, n, cyc)) return "non-manifold vertex fan";
        N = (int)cyc.size() / 2;
        for (int i = 1; i < 2 * N; ++i)
            if (!add_flux(n, cyc[i - 1], cyc[i], i / (2.0 * N) - 0.5)) return "BC construction failed (source fan)";
    }
    m.bc_ptr.assign(m.nf + 1, 0);
    for (auto& kv : flux) m.bc_ptr[kv.first.first + 1]++;
    for (int t = 0; t < m.nf; ++t) m.bc_ptr[t + 1] += m.bc_ptr[t];
    m.bc_fn.resize(flux.size());
    m.bc_phi.resize(3 * flux.size());
    std::vector<int> fill(m.bc_ptr.begin(), m.bc_ptr.end() - 1);
    for (auto& kv : flux) {   // map order: by fine triangle, then function index
        const int t = kv.first.first, pos = fill[t]++;
        m.bc_fn[pos] = kv.first.second;
        for (int k = 0; k < 3; ++k) m.bc_phi[3 * pos + k] = kv.second[k];
    }
    return "";
}

void gauss_legendre(int n, double* x, double* w) {
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < n; ++i) {
        double z = std::cos(pi * (i + 0.75) / (n + 0.5)), dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) { const double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k; p0 = p1; p1 = p2; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) { const double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k; p0 = p1; p1 = p2; }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[n - 1 - i] = z;
        w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

}  // namespace tdc
