"""Seeded plane-wave excitation parameters (shared inputs; no method arithmetic).

A plane wave is described by its direction k (unit), polarisation p (unit,
orthogonal to k), amplitude A, arrival time t0 and Gaussian width sigma:
    e_in(r, t) = A p exp(-((t - k.r - t0) / sigma)^2),   h_in = k x e_in
(natural units c = eta = 1).  This module only produces the parameter arrays.
"""
from __future__ import annotations

import numpy as np


def single(k=(0.0, 0.0, 1.0), p=(1.0, 0.0, 0.0), amp=1.0, t0=8.0, sigma=2.0):
    """One plane wave as (R=1) parameter arrays."""
    return {
        "k": np.asarray([k], dtype=np.float64),
        "p": np.asarray([p], dtype=np.float64),
        "amp": np.asarray([amp], dtype=np.float64),
        "t0": np.asarray([t0], dtype=np.float64),
        "sigma": np.asarray([sigma], dtype=np.float64),
    }


def fibonacci_directions(n: int) -> np.ndarray:
    """n unit directions on a Fibonacci sphere: z_i = 1-(2i+1)/n, phi_i = i*pi*(3-sqrt 5)."""
    i = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / n
    phi = i * np.pi * (3.0 - 5.0 ** 0.5)
    s = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([s * np.cos(phi), s * np.sin(phi), z], axis=1)


def seeded_polarisations(k: np.ndarray, seed: int) -> np.ndarray:
    """Normal draws (numpy PCG64) made orthogonal to each k and normalised."""
    rng = np.random.Generator(np.random.PCG64(seed))
    g = rng.standard_normal(size=k.shape)
    g = g - np.sum(g * k, axis=1, keepdims=True) * k
    return g / np.linalg.norm(g, axis=1, keepdims=True)


def fibonacci_batch(n: int, seed: int, t0: float = 8.0, sigma: float = 1.0, amp: float = 1.0):
    k = fibonacci_directions(n)
    return {
        "k": k,
        "p": seeded_polarisations(k, seed),
        "amp": np.full(n, amp, dtype=np.float64),
        "t0": np.full(n, t0, dtype=np.float64),
        "sigma": np.full(n, sigma, dtype=np.float64),
    }


def random_batch(n: int, seed: int, t0: float = 8.0, sigma: float = 2.0):
    """n seeded random directions (uniform on the sphere) with seeded orthogonal polarisations."""
    rng = np.random.Generator(np.random.PCG64(seed))
    k = rng.standard_normal(size=(n, 3))
    k /= np.linalg.norm(k, axis=1, keepdims=True)
    return {
        "k": k,
        "p": seeded_polarisations(k, seed + 1),
        "amp": np.ones(n),
        "t0": np.full(n, t0),
        "sigma": np.full(n, sigma),
    }


def as_arrays(pw: dict):
    """Contiguous float64 arrays in the order the C-ABI expects: k (R x 3), p (R x 3), amp, t0, sigma."""
    return tuple(np.ascontiguousarray(pw[key], dtype=np.float64) for key in ("k", "p", "amp", "t0", "sigma"))
