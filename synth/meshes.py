"""Seeded synthetic surface meshes (shared inputs for the oracle and the CUDA path).

This module only generates geometry: vertex coordinates (float64, N_V x 3) and
triangles (int32, N_C x 3), each triangle listed counter-clockwise when seen
from outside the closed surface (outward normal by the right-hand rule).  It
holds none of the method's arithmetic.

Workloads (the paper's own meshes are not available; these stand in for them):
  * icosphere(level)      -- icosahedron, 1->4 midpoint subdivision, projected
                             to the unit sphere after every level
                             (level 2: 320 triangles / 480 edges,
                              level 4: 5120 triangles / 7680 edges).
  * octasphere(level)     -- octahedron, same subdivision (level 5: 8192 / 12288).
  * ellipsoid(level, a)   -- octasphere scaled by the semi-axes a.
  * torus(R, r, nu, nv)   -- (nu x nv) parametric grid, each quad split on the
                             (i,j)-(i+1,j+1) diagonal (24 x 12: 576 / 864).
"""
from __future__ import annotations

import numpy as np


def _subdivide(V: list, F: np.ndarray, project: bool) -> tuple[list, np.ndarray]:
    """Split every triangle into four through its edge midpoints."""
    mid: dict[tuple[int, int], int] = {}

    def midpoint(a: int, b: int) -> int:
        key = (a, b) if a < b else (b, a)
        idx = mid.get(key)
        if idx is None:
            p = 0.5 * (V[a] + V[b])
            if project:
                p = p / np.linalg.norm(p)
            idx = len(V)
            V.append(p)
            mid[key] = idx
        return idx

    out = []
    for a, b, c in F.tolist():
        ab, bc, ca = midpoint(a, b), midpoint(b, c), midpoint(c, a)
        out += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
    return V, np.asarray(out, dtype=np.int32)


def _orient_outward(V: np.ndarray, F: np.ndarray, centre: np.ndarray) -> np.ndarray:
    """Flip triangles whose right-hand normal points towards `centre` (star-shaped surfaces)."""
    F = F.copy()
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    n = np.cross(b - a, c - a)
    g = (a + b + c) / 3.0 - centre
    flip = np.einsum("ij,ij->i", n, g) < 0
    F[flip] = F[flip][:, [0, 2, 1]]
    return F


def icosahedron() -> tuple[np.ndarray, np.ndarray]:
    t = (1.0 + 5.0 ** 0.5) / 2.0
    V = np.array(
        [[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
         [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
         [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]], dtype=np.float64)
    V /= np.linalg.norm(V, axis=1, keepdims=True)
    F = np.array(
        [[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
         [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
         [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
         [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int32)
    return V, _orient_outward(V, F, np.zeros(3))


def octahedron() -> tuple[np.ndarray, np.ndarray]:
    V = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]],
                 dtype=np.float64)
    F = np.array([[0, 2, 4], [2, 1, 4], [1, 3, 4], [3, 0, 4],
                  [2, 0, 5], [1, 2, 5], [3, 1, 5], [0, 3, 5]], dtype=np.int32)
    return V, _orient_outward(V, F, np.zeros(3))


def tetrahedron() -> tuple[np.ndarray, np.ndarray]:
    V = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=np.float64) / 3 ** 0.5
    F = np.array([[0, 1, 2], [0, 2, 3], [0, 3, 1], [1, 3, 2]], dtype=np.int32)
    return V, _orient_outward(V, F, np.zeros(3))


def _sphere_from(base, level: int):
    V, F = base()
    Vl = list(V)
    for _ in range(level):
        Vl, F = _subdivide(Vl, F, project=True)
    V = np.asarray(Vl, dtype=np.float64)
    return V, _orient_outward(V, F, np.zeros(3))


def icosphere(level: int) -> tuple[np.ndarray, np.ndarray]:
    """Unit sphere from the icosahedron, `level` midpoint subdivisions, projected each level."""
    return _sphere_from(icosahedron, level)


def octasphere(level: int) -> tuple[np.ndarray, np.ndarray]:
    """Unit sphere from the octahedron, `level` midpoint subdivisions, projected each level."""
    return _sphere_from(octahedron, level)


def ellipsoid(level: int, semi_axes=(2.0, 1.0, 0.5)) -> tuple[np.ndarray, np.ndarray]:
    """Octasphere scaled to the given semi-axes (orientation is preserved by a positive scaling)."""
    V, F = octasphere(level)
    return V * np.asarray(semi_axes, dtype=np.float64)[None, :], F


def torus(R: float = 1.0, r: float = 0.4, nu: int = 24, nv: int = 12) -> tuple[np.ndarray, np.ndarray]:
    """Torus of major radius R and minor radius r on an (nu x nv) grid, outward oriented."""
    u = 2.0 * np.pi * np.arange(nu) / nu
    v = 2.0 * np.pi * np.arange(nv) / nv
    V = np.empty((nu * nv, 3), dtype=np.float64)
    for i in range(nu):
        for j in range(nv):
            rho = R + r * np.cos(v[j])
            V[i * nv + j] = (rho * np.cos(u[i]), rho * np.sin(u[i]), r * np.sin(v[j]))
    F = []
    for i in range(nu):
        for j in range(nv):
            a = i * nv + j
            b = ((i + 1) % nu) * nv + j
            c = ((i + 1) % nu) * nv + (j + 1) % nv
            d = i * nv + (j + 1) % nv
            F += [(a, b, c), (a, c, d)]
    F = np.asarray(F, dtype=np.int32)
    # outward = away from the tube's centre circle
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    n = np.cross(b - a, c - a)
    g = (a + b + c) / 3.0
    ring = g.copy()
    ring[:, 2] = 0.0
    ring *= (R / np.linalg.norm(ring, axis=1))[:, None]
    flip = np.einsum("ij,ij->i", n, g - ring) < 0
    F[flip] = F[flip][:, [0, 2, 1]]
    return V, F


def perturbed(V: np.ndarray, F: np.ndarray, amplitude: float, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """Seeded radial jitter of the vertices (keeps connectivity); used for irregular test meshes."""
    rng = np.random.Generator(np.random.PCG64(seed))
    s = 1.0 + amplitude * rng.uniform(-1.0, 1.0, size=(V.shape[0], 1))
    return V * s, F.copy()
