"""Far field of a marched surface current at one frequency, and the low-frequency (Rayleigh) far
field of a PEC sphere: the large-time-step accuracy test of Sec. V (the sphere marched with a time
step about 10^5 times its light-crossing time; its far field at 3 Hz compared with Mie).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Units c = eta = mu = eps = 1 (times in metres of light travel), phasors e^{j w t}, spectra
F(w) = int f(t) e^{-j w t} dt, wavenumber k = w.
  Current spectrum. The march's output j_i (Eq. post_processing) are the coefficients of the hat
  basis h_i(t) = h_0(t - t_i), t_i = i dt (i = 1..Nt), whose spectrum is dt sinc^2(w dt / 2):
      J_m(w) = dt sinc^2(w dt / 2) sum_i j_m[i] e^{-j w t_i}.
  Radiation vector and far-field amplitude (the scattered field is F(rhat) e^{-j k r} / r):
      N(rhat) = sum_m J_m(w) int f_m(r') e^{j k rhat.r'} dS',
      F(rhat) = -j k / (4 pi) (I - rhat rhat) N(rhat).
  The integral over each triangle of f_m uses the 7-point degree-5 rule (f_m is linear; at the
  test's k D ~ 1e-7 the phase is linear to 1e-14).
  Rayleigh limit (k a -> 0) for a PEC sphere of radius a in E0 e^{-j k khat.r}, H0 = khat x E0:
  induced dipoles p = 4 pi a^3 E0 and m = -2 pi a^3 H0 (the textbook small-sphere result), whose
  far field is
      F(rhat) = k^2 / (4 pi) [ (I - rhat rhat) p - rhat x m ] = k^2 a^3 [ (I - rhat rhat) E0 + rhat x H0 / 2 ].
  Its E-plane pattern is |cos(theta) - 1/2|, its H-plane pattern |1 - cos(theta)/2|.
  Incident amplitude at the origin for the pulse amp p exp(-((t - khat.r - t0)/sigma)^2):
      E0(w) = amp p sigma sqrt(pi) exp(-(w sigma / 2)^2) e^{-j w t0}.
"""
from __future__ import annotations

import numpy as np

from .rhs import _R7_L, _R7_W


def current_spectrum(j: np.ndarray, dt: float, w: float) -> np.ndarray:
    """J_m(w) for j (Nt, ne, R) at t_i = i dt, i = 1..Nt: (ne, R) complex."""
    nt = j.shape[0]
    t = dt * np.arange(1, nt + 1)
    x = 0.5 * w * dt
    hat = dt * (np.sin(x) / x) ** 2 if x != 0.0 else dt
    return hat * np.einsum("i,imr->mr", np.exp(-1j * w * t), j)


def radiation_integrals(topo, rhat: np.ndarray, k: float) -> np.ndarray:
    """int f_m(r) e^{j k rhat.r} dS for every edge m and direction: (ndir, ne, 3) complex."""
    rhat = np.atleast_2d(rhat)
    out = np.zeros((rhat.shape[0], topo.ne, 3), dtype=complex)
    for m in range(topo.ne):
        for c in (topo.cplus[m], topo.cminus[m]):
            tri = topo.V[topo.F[c]]
            pts = _R7_L @ tri                                   # (7, 3)
            f = topo.rwg(m, c, pts)                             # (7, 3)
            ph = np.exp(1j * k * (pts @ rhat.T))                # (7, ndir)
            out[:, m, :] += topo.area[c] * np.einsum("q,qd,qx->dx", _R7_W, ph, f)
    return out


def far_field(topo, j: np.ndarray, dt: float, k: float, rhat: np.ndarray) -> np.ndarray:
    """F(rhat) of the marched currents j (Nt, ne, R): (ndir, R, 3) complex."""
    rhat = np.atleast_2d(rhat)
    Jw = current_spectrum(j, dt, k)                             # (ne, R)
    N = np.einsum("dmx,mr->drx", radiation_integrals(topo, rhat, k), Jw)
    proj = np.eye(3)[None] - rhat[:, :, None] * rhat[:, None, :]
    return -1j * k / (4.0 * np.pi) * np.einsum("dxy,dry->drx", proj, N)


def incident_amplitude(pw: dict, r: int, w: float) -> np.ndarray:
    """E0(w) of wave r at the origin: (3,) complex."""
    s = pw["sigma"][r]
    g = s * np.sqrt(np.pi) * np.exp(-(0.5 * w * s) ** 2) * np.exp(-1j * w * pw["t0"][r])
    return pw["amp"][r] * g * np.asarray(pw["p"][r], dtype=float)


def rayleigh_sphere(rhat: np.ndarray, k: float, a: float, E0: np.ndarray, khat: np.ndarray) -> np.ndarray:
    """Far-field amplitude of a small PEC sphere: (ndir, 3) complex."""
    rhat = np.atleast_2d(rhat)
    H0 = np.cross(khat, E0)
    proj = np.eye(3)[None] - rhat[:, :, None] * rhat[:, None, :]
    return k * k * a ** 3 * (np.einsum("dxy,y->dx", proj, E0) + 0.5 * np.cross(rhat, H0[None, :]))
