"""Mesh topology of the oracle: edges, RWG supports, Lambda and Sigma (Sec. II-C, II-D).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Readings of the paper fixed here:
  * edges are the unique unordered vertex pairs, numbered in lexicographic order of
    (min v, max v); the edge is oriented v- = min -> v+ = max (Sec. II-D orientation of Lambda);
  * c+ of an edge is the triangle whose counter-clockwise cycle (about the outward
    normal) runs v- -> v+, c- the other one (Sec. II-D, definition of Sigma); with this
    pairing Sigma^T Lambda = 0 and RWG loops are divergence-free;
  * RWG f_n (Sec. II-C, Fig. 1) in the paper's normalisation without edge length:
    (r - r+)/(2 A+) on c+, (r- - r)/(2 A-) on c-, i.e. unit flux c+ -> c-;
  * D = largest vertex-to-vertex distance; T0 = D / c.
"""
from __future__ import annotations

import numpy as np


class Topology:
    def __init__(self, V: np.ndarray, F: np.ndarray):
        V = np.ascontiguousarray(V, dtype=np.float64)
        F = np.ascontiguousarray(F, dtype=np.int32)
        self.V, self.F = V, F
        self.nv, self.nc = V.shape[0], F.shape[0]
        # unique edges in lexicographic order
        pairs = set()
        for a, b, c in F.tolist():
            for x, y in ((a, b), (b, c), (c, a)):
                pairs.add((min(x, y), max(x, y)))
        E = np.array(sorted(pairs), dtype=np.int32)
        self.E = E
        self.ne = E.shape[0]
        index = {tuple(e): i for i, e in enumerate(E.tolist())}
        cplus = -np.ones(self.ne, dtype=np.int32)
        cminus = -np.ones(self.ne, dtype=np.int32)
        ropp_plus = -np.ones(self.ne, dtype=np.int32)
        ropp_minus = -np.ones(self.ne, dtype=np.int32)
        tedge = np.zeros((self.nc, 3), dtype=np.int32)
        tsign = np.zeros((self.nc, 3), dtype=np.float64)
        count = np.zeros(self.ne, dtype=np.int32)
        for c, tri in enumerate(F.tolist()):
            for j in range(3):
                a, b = tri[(j + 1) % 3], tri[(j + 2) % 3]      # edge opposite local vertex j, CCW a->b
                m = index[(min(a, b), max(a, b))]
                count[m] += 1
                tedge[c, j] = m
                if a < b:           # traversal v- -> v+ : this triangle is c+
                    if cplus[m] != -1:
                        raise ValueError("inconsistent orientation or non-manifold edge")
                    cplus[m], ropp_plus[m] = c, tri[j]
                    tsign[c, j] = 1.0
                else:
                    if cminus[m] != -1:
                        raise ValueError("inconsistent orientation or non-manifold edge")
                    cminus[m], ropp_minus[m] = c, tri[j]
                    tsign[c, j] = -1.0
        if np.any(count != 2) or np.any(cplus < 0) or np.any(cminus < 0):
            raise ValueError("mesh is not a closed consistently oriented 2-manifold")
        self.cplus, self.cminus = cplus, cminus
        self.ropp_plus, self.ropp_minus = ropp_plus, ropp_minus
        self.tedge, self.tsign = tedge, tsign
        # vertex valence (number of triangles at each vertex = number of edges for a closed mesh)
        self.valence = np.bincount(F.reshape(-1), minlength=self.nv).astype(np.int32)
        chi = self.nv - self.ne + self.nc
        self.genus = (2 - chi) // 2
        self._check_connected()
        a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
        cr = np.cross(b - a, c - a)
        self.area = 0.5 * np.linalg.norm(cr, axis=1)
        self.normal = cr / (2.0 * self.area)[:, None]
        # diameter: largest vertex-to-vertex distance
        D = 0.0
        for i in range(self.nv):
            D = max(D, float(np.max(np.linalg.norm(V - V[i], axis=1))))
        self.D = D

    def _check_connected(self):
        parent = list(range(self.nc))

        def find(x):
            while parent[x] != x:
                parent[x] = parent[parent[x]]
                x = parent[x]
            return x

        for m in range(self.ne):
            a, b = find(int(self.cplus[m])), find(int(self.cminus[m]))
            if a != b:
                parent[a] = b
        if len({find(i) for i in range(self.nc)}) != 1:
            raise ValueError("mesh is not connected")

    def Lambda(self) -> np.ndarray:
        """Vertex-edge incidence Lambda (N_E x N_V): +1 at v+, -1 at v- (Sec. II-D)."""
        L = np.zeros((self.ne, self.nv), dtype=np.int64)
        L[np.arange(self.ne), self.E[:, 1]] = 1
        L[np.arange(self.ne), self.E[:, 0]] = -1
        return L

    def Sigma(self) -> np.ndarray:
        """Face-edge incidence Sigma (N_E x N_C): +1 at c+, -1 at c- (Sec. II-D)."""
        S = np.zeros((self.ne, self.nc), dtype=np.int64)
        S[np.arange(self.ne), self.cplus] = 1
        S[np.arange(self.ne), self.cminus] = -1
        return S

    def rwg(self, m: int, c: int, r: np.ndarray) -> np.ndarray:
        """Evaluate f_m at points r (n x 3) lying in triangle c (Sec. II-C, Fig. 1)."""
        if c == self.cplus[m]:
            return (r - self.V[self.ropp_plus[m]]) / (2.0 * self.area[c])
        if c == self.cminus[m]:
            return (self.V[self.ropp_minus[m]] - r) / (2.0 * self.area[c])
        return np.zeros_like(r)


def n_lags(D: float, dt: float, order: int = 1) -> int:
    """Number of time blocks T_0..T_{K-1}: T_k vanishes once (k - order - 1) dt >= D (q_0 is
    supported on [-dt, (order + 1) dt])."""
    return int(np.ceil(D / dt + order + 1.0))
