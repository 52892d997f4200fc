"""Barycentric refinement and Buffa-Christiansen functions of the oracle (Sec. II-C, Fig. 2).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper defines g_n only as "a linear combination of RWG functions on the
barycentric refinement with the coefficients of [BC2007]" (Sec. II-C).  Reading used
here (written in terms of fluxes of unit-flux fine RWG functions):
  * each coarse triangle (a, b, c) is split into 6 fine triangles by its barycentre
    and edge midpoints; every fine triangle has exactly one coarse vertex;
  * the dual cell D_v of a coarse vertex v is the set of its 2 N_v fine triangles
    (N_v = number of coarse triangles at v);
  * g_n carries unit flux from D_{v+} to D_{v-} across the dual edge of e_n
    (the fine edges midpoint->barycentre of c+ and of c-, 1/2 each); inside each cell the
    flux through the radial fine edges falls linearly by 1/(2 N_v) per fine triangle
    ((N_v - i)/(2 N_v) pattern), with zero flux through the coarse half-edge of e_n;
  * hence every fine triangle of D_{v+} carries charge +1/(2 N_{v+}) and every fine
    triangle of D_{v-} charge -1/(2 N_{v-}): div g_n = sum_v Lambda_{nv} rho_v.
With this sign n x g_n points from c+ to c- like f_n, so G_nn > 0.

Representation: on a fine triangle t with vertices (w0, w1, w2) and area A,
g_n(r) = sum_j phi_{n,t,j} (r - w_j) / (2 A), phi = outward flux through the fine edge
opposite w_j.  Stored as a CSR over fine triangles (bc_ptr, bc_fn, bc_phi).
"""
from __future__ import annotations

import numpy as np

from .topology import Topology


class BarycentricBC:
    def __init__(self, topo: Topology):
        self.topo = topo
        nv, ne, nc = topo.nv, topo.ne, topo.nc
        V, F = topo.V, topo.F
        # fine vertices: coarse vertices, edge midpoints, barycentres
        mids = 0.5 * (V[topo.E[:, 0]] + V[topo.E[:, 1]])
        bary = (V[F[:, 0]] + V[F[:, 1]] + V[F[:, 2]]) / 3.0
        self.fV = np.ascontiguousarray(np.concatenate([V, mids, bary], axis=0))
        fF, fparent, fvert, fmid = [], [], [], []
        # ft[(c, u, m)] = fine triangle in coarse c with coarse vertex u and midpoint of edge m
        self.ft = {}
        for c, tri in enumerate(F.tolist()):
            b = nv + ne + c
            for j in range(3):
                u = tri[j]
                # the two coarse edges of c at u: opposite local vertices j+1 and j+2
                e_next = int(topo.tedge[c, (j + 2) % 3])   # edge (u, tri[j+1])
                e_prev = int(topo.tedge[c, (j + 1) % 3])   # edge (tri[j+2], u)
                # CCW fine triangles with u first: (u, m_next, b) and (u, b, m_prev)
                for m, verts in ((e_next, (u, nv + e_next, b)), (e_prev, (u, b, nv + e_prev))):
                    self.ft[(c, u, m)] = len(fF)
                    fF.append(verts)
                    fparent.append(c)
                    fvert.append(u)
                    fmid.append(m)
        self.fF = np.asarray(fF, dtype=np.int32)
        self.fparent = np.asarray(fparent, dtype=np.int32)
        self.fvert = np.asarray(fvert, dtype=np.int32)
        self.fmid = np.asarray(fmid, dtype=np.int32)
        self.nf = self.fF.shape[0]
        a, b_, c_ = (self.fV[self.fF[:, i]] for i in range(3))
        cr = np.cross(b_ - a, c_ - a)
        self.farea = 0.5 * np.linalg.norm(cr, axis=1)
        self._build_functions()

    # ------------------------------------------------------------------
    def _local_edge(self, t: int, p: int, q: int) -> int:
        """Local index j of fine triangle t whose opposite edge is {p, q}."""
        tri = self.fF[t].tolist()
        for j in range(3):
            if {tri[(j + 1) % 3], tri[(j + 2) % 3]} == {p, q}:
                return j
        raise KeyError("edge not in triangle")

    def _shared(self, ta: int, tb: int):
        s = set(self.fF[ta].tolist()) & set(self.fF[tb].tolist())
        if len(s) != 2:
            raise KeyError("fine triangles are not adjacent")
        return tuple(s)

    def _flux(self, coef: dict, n: int, ta: int, tb: int, phi: float):
        """Add flux phi from fine triangle ta to fine triangle tb through their common edge."""
        if phi == 0.0:
            return
        p, q = self._shared(ta, tb)
        ja, jb = self._local_edge(ta, p, q), self._local_edge(tb, p, q)
        coef.setdefault((ta, n), np.zeros(3))[ja] += phi
        coef.setdefault((tb, n), np.zeros(3))[jb] -= phi

    def _cycle(self, v: int, c_start: int, m_start: int):
        """Fine triangles around coarse vertex v, starting at the one in c_start next to the
        half-edge (v, mid m_start) and walking away from that half-edge."""
        topo = self.topo
        out = []
        c, m = c_start, m_start
        while True:
            out.append(self.ft[(c, v, m)])
            # the other coarse edge of c at v
            tri = topo.F[c].tolist()
            j = tri.index(v)
            e1, e2 = int(topo.tedge[c, (j + 1) % 3]), int(topo.tedge[c, (j + 2) % 3])
            m2 = e1 if e2 == m else e2
            out.append(self.ft[(c, v, m2)])
            c2 = int(topo.cminus[m2]) if topo.cplus[m2] == c else int(topo.cplus[m2])
            c, m = c2, m2
            if m == m_start:
                break
        return out

    def _build_functions(self):
        topo = self.topo
        coef: dict = {}
        for n in range(topo.ne):
            vm, vp = int(topo.E[n, 0]), int(topo.E[n, 1])
            cp, cm = int(topo.cplus[n]), int(topo.cminus[n])
            # across the dual edge: 1/2 through (mid, bary c+) and 1/2 through (mid, bary c-)
            for c in (cp, cm):
                self._flux(coef, n, self.ft[(c, vp, n)], self.ft[(c, vm, n)], 0.5)
            # sink cell D_{v-}: flux (1/2 - i/(2N)) from t_i to t_{i+1}
            cyc = self._cycle(vm, cp, n)
            N = len(cyc) // 2
            for i in range(1, 2 * N):
                self._flux(coef, n, cyc[i - 1], cyc[i], 0.5 - i / (2.0 * N))
            # source cell D_{v+}: flux (i/(2N) - 1/2) from t_i to t_{i+1}
            cyc = self._cycle(vp, cp, n)
            N = len(cyc) // 2
            for i in range(1, 2 * N):
                self._flux(coef, n, cyc[i - 1], cyc[i], i / (2.0 * N) - 0.5)
        # CSR over fine triangles
        per_t: list = [[] for _ in range(self.nf)]
        for (t, n), phi in coef.items():
            per_t[t].append((n, phi))
        ptr, fn, ph = [0], [], []
        for t in range(self.nf):
            for n, phi in sorted(per_t[t], key=lambda z: z[0]):
                fn.append(n)
                ph.append(phi)
            ptr.append(len(fn))
        self.bc_ptr = np.asarray(ptr, dtype=np.int32)
        self.bc_fn = np.asarray(fn, dtype=np.int32)
        self.bc_phi = np.ascontiguousarray(np.asarray(ph, dtype=np.float64).reshape(-1, 3))

    # ------------------------------------------------------------------
    def eval(self, n: int, t: int, r: np.ndarray) -> np.ndarray:
        """g_n at points r (k x 3) in fine triangle t."""
        out = np.zeros_like(r)
        for e in range(self.bc_ptr[t], self.bc_ptr[t + 1]):
            if self.bc_fn[e] != n:
                continue
            for j in range(3):
                w = self.fV[self.fF[t, j]]
                out += self.bc_phi[e, j] * (r - w) / (2.0 * self.farea[t])
        return out

    def charges(self) -> np.ndarray:
        """Net outward flux (= total charge) of every (BC function, fine triangle) pair: nf x ne."""
        Q = np.zeros((self.nf, self.topo.ne))
        for t in range(self.nf):
            for e in range(self.bc_ptr[t], self.bc_ptr[t + 1]):
                Q[t, self.bc_fn[e]] += self.bc_phi[e].sum()
        return Q
