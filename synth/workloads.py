"""The five synthetic workloads of the hot path, by name and size (shared inputs only).

Each workload is a dict: mesh (V, F), time step dt, number of steps Nt,
coupling alpha and the plane-wave batch.  Names state what they are:

  sphere480_fp64     icosphere level 2 (320 tri / 480 edges), dt 0.2, 300 steps, x-pol along +z,
                     sigma 2, t0 8; FP64 path, direct solve.
  torus864_fp32      torus R 1, r 0.4, 24x12 (576 tri / 864 edges), genus 1, dt 2.0, 1000 steps,
                     same pulse; FP32 history.
  sphere7680_r64     icosphere level 4 (5120 tri / 7680 edges), 64 Fibonacci directions with seeded
                     orthogonal polarisations (seed 2312063670), sigma 1, t0 8, dt 0.05, 2000 steps;
                     split-precision tensor-core history (fp16 hi/lo with power-of-two scaling, which
                     meets 1e-5; bf16 hi/lo selectable).
  sphere1920_r64     the same at icosphere level 3 (1280 tri / 1920 edges): a smaller case of the
                     same tensor-core kernels whose blocks (634 MB) still exceed the L2 cache.
  ellipsoid12288     octasphere level 5 scaled to semi-axes (2, 1, 0.5) (8192 tri / 12288 edges),
                     dt 0.1, 1500 steps, GMRES tol 1e-8 (learned initial guess).
  sphere7680_train8  icosphere level 4, dt 0.1, 300 steps, 8 Fibonacci directions (seed 2312063671),
                     sigma 2: trajectories that train the learned GMRES guess.
  batch_uneven       the first 16 scatterers of the batch32 family with at most 3456 edges.
  batch32            32 seeded scatterers (spheres, ellipsoids, tori) of 480..12288 edges, dt 0.2,
                     1000 steps, one direction each.
"""
from __future__ import annotations

import numpy as np

from . import excitation, meshes


def sphere480_fp64():
    V, F = meshes.icosphere(2)
    return dict(name="sphere480_fp64", V=V, F=F, dt=0.2, Nt=300, alpha=1.0,
                pw=excitation.single(t0=8.0, sigma=2.0), precision="fp64")


def torus864_fp32():
    V, F = meshes.torus(1.0, 0.4, 24, 12)
    return dict(name="torus864_fp32", V=V, F=F, dt=2.0, Nt=1000, alpha=1.0,
                pw=excitation.single(t0=8.0, sigma=2.0), precision="fp32")


def sphere7680_r64(n_dir: int = 64, precision: str = "fp16x3"):
    V, F = meshes.icosphere(4)
    return dict(name="sphere7680_r64", V=V, F=F, dt=0.05, Nt=2000, alpha=1.0,
                pw=excitation.fibonacci_batch(n_dir, seed=2312063670, t0=8.0, sigma=1.0),
                precision=precision)


def sphere1920_r64(n_dir: int = 64, precision: str = "fp16x3"):
    V, F = meshes.icosphere(3)
    return dict(name="sphere1920_r64", V=V, F=F, dt=0.05, Nt=2000, alpha=1.0,
                pw=excitation.fibonacci_batch(n_dir, seed=2312063670, t0=8.0, sigma=1.0),
                precision=precision)


def ellipsoid12288():
    V, F = meshes.ellipsoid(5, (2.0, 1.0, 0.5))
    return dict(name="ellipsoid12288", V=V, F=F, dt=0.1, Nt=1500, alpha=1.0,
                pw=excitation.single(t0=8.0, sigma=2.0), precision="fp32", solver="gmres",
                gmres_tol=1e-8)


def sphere7680_train8():
    """Training trajectories for the learned GMRES guess: the 7680-edge sphere, dt 0.1, 8 Fibonacci
    directions with seeded polarisations, the same pulse width as the ellipsoid evaluation."""
    V, F = meshes.icosphere(4)
    return dict(name="sphere7680_train8", V=V, F=F, dt=0.1, Nt=300, alpha=1.0,
                pw=excitation.fibonacci_batch(8, seed=2312063671, t0=8.0, sigma=2.0), precision="fp32")


def _family(seed: int):
    """Endless seeded sequence of scatterers: sphere, ellipsoid (semi-axes U[0.5, 2]) or torus
    (R 1, r U[0.2, 0.5]) from size menus of 480..12288 edges; one random plane wave each."""
    rng = np.random.Generator(np.random.PCG64(seed))
    s = 0
    while True:
        fam = int(rng.integers(0, 3))
        if fam == 0:
            lvl = int(rng.integers(2, 5))              # icosphere 480 / 1920 / 7680 edges
            V, F = meshes.icosphere(lvl)
        elif fam == 1:
            lvl = int(rng.integers(3, 6))              # octasphere 768 / 3072 / 12288 edges
            ax = rng.uniform(0.5, 2.0, size=3)
            V, F = meshes.ellipsoid(lvl, tuple(ax))
        else:
            nv = int(rng.choice([8, 12, 16, 24, 32]))
            nu = int(rng.choice([2, 4])) * nv
            rr = float(rng.uniform(0.2, 0.5))
            V, F = meshes.torus(1.0, rr, nu, nv)
        pw = excitation.random_batch(1, seed=seed + 1000 + s, t0=8.0, sigma=2.0)
        yield dict(name=f"batch32_{s}", V=V, F=F, dt=0.2, Nt=1000, alpha=1.0, pw=pw, precision="fp32")
        s += 1


def batch32(seed: int = 2312063675, n: int = 32):
    """32 seeded scatterers from size menus (edges 480..12288)."""
    g = _family(seed)
    return [next(g) for _ in range(n)]


def batch_uneven(n: int = 16, max_edges: int = 3456, seed: int = 2312063675):
    """The first n scatterers of the same seeded family with at most max_edges edges (uneven sizes
    whose assembly fits a short run)."""
    out = []
    for p in _family(seed):
        if p["F"].shape[0] * 3 // 2 <= max_edges:
            out.append(p)
        if len(out) == n:
            return out


def small_sphere(level: int = 1, dt: float = 0.4, Nt: int = 40):
    """Small icosphere case the oracle finishes in seconds (80 tri / 120 edges at level 1)."""
    V, F = meshes.icosphere(level)
    return dict(name=f"icosphere{level}", V=V, F=F, dt=dt, Nt=Nt, alpha=1.0,
                pw=excitation.single(t0=8.0, sigma=2.0), precision="fp64")


def small_torus(nu: int = 8, nv: int = 4, dt: float = 0.5, Nt: int = 40):
    V, F = meshes.torus(1.0, 0.4, nu, nv)
    return dict(name=f"torus{nu}x{nv}", V=V, F=F, dt=dt, Nt=Nt, alpha=1.0,
                pw=excitation.single(t0=8.0, sigma=2.0), precision="fp64")
