"""Incident-field tests of the oracle (Sec. II-C right-hand sides, Sec. V excitation).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

  e_m(t) = <n x f_m, n x e_in(t)> = int f_m . e_in         (7-point rule on coarse triangles)
  h_m(t) = <n x g_m, n x h_in(t)> = int g_m . h_in         (3-point rule on fine triangles)
  e_in(r, t) = A p exp(-((t - k.r - t0)/sigma)^2),  h_in = k x e_in   (c = eta = 1)
Reading: the configs' pulse form (amplitude A, width sigma) replaces the paper's
4A/(w sqrt(pi)) and 4/w parametrisation; with w = 8 the paper's sigma is 2.
"""
from __future__ import annotations

import numpy as np

_R7_L = np.array([
    [1 / 3, 1 / 3, 1 / 3],
    [0.05971587178976982, 0.47014206410511511, 0.47014206410511511],
    [0.47014206410511511, 0.05971587178976982, 0.47014206410511511],
    [0.47014206410511511, 0.47014206410511511, 0.05971587178976982],
    [0.79742698535308731, 0.10128650732345634, 0.10128650732345634],
    [0.10128650732345634, 0.79742698535308731, 0.10128650732345634],
    [0.10128650732345634, 0.10128650732345634, 0.79742698535308731]])
_R7_W = np.array([0.225] + [0.13239415278850619] * 3 + [0.12593918054482714] * 3)
_R3_L = np.array([[2 / 3, 1 / 6, 1 / 6], [1 / 6, 2 / 3, 1 / 6], [1 / 6, 1 / 6, 2 / 3]])
_R3_W = np.full(3, 1 / 3)


def _envelope(pts: np.ndarray, times: np.ndarray, pw: dict, r: int) -> np.ndarray:
    """A exp(-((t - k.r - t0)/sigma)^2) at all (time, point) pairs: (Nt, npts)."""
    arg = (times[:, None] - (pts @ pw["k"][r])[None, :] - pw["t0"][r]) / pw["sigma"][r]
    return pw["amp"][r] * np.exp(-arg * arg)


def incident_tests(ops, pw: dict, times: np.ndarray):
    """e (Nt, ne, R) and h (Nt, ne, R) at the given times."""
    t, b = ops.topo, ops.bc
    times = np.asarray(times, dtype=np.float64)
    R = pw["k"].shape[0]
    e = np.zeros((len(times), t.ne, R))
    h = np.zeros((len(times), t.ne, R))
    for c in range(t.nc):
        w = t.V[t.F[c]]
        pts = _R7_L @ w
        wts = _R7_W * t.area[c]
        for r in range(R):
            env = _envelope(pts, times, pw, r)                       # (Nt, 7)
            for j in range(3):
                f = t.tsign[c, j] * (pts - w[j]) / (2.0 * t.area[c])
                e[:, t.tedge[c, j], r] += env @ (wts * (f @ pw["p"][r]))
    for ft in range(b.nf):
        w = b.fV[b.fF[ft]]
        pts = _R3_L @ w
        wts = _R3_W * b.farea[ft]
        for r in range(R):
            env = _envelope(pts, times, pw, r)
            hdir = np.cross(pw["k"][r], pw["p"][r])                 # h_in = k x e_in
            for q in range(b.bc_ptr[ft], b.bc_ptr[ft + 1]):
                g = np.zeros((3, 3))
                for j in range(3):
                    g += b.bc_phi[q, j] * (pts - w[j]) / (2.0 * b.farea[ft])
                h[:, b.bc_fn[q], r] += env @ (wts * (g @ hdir))
    return e, h
