"""Helpers of the Mie-series physics pins (test infrastructure): the PEC-sphere series in the
exp(-i w t) convention of vector spherical wave functions, its Fourier synthesis for a Gaussian
pulse, and the evaluation of an RWG-expanded current at points of the unit sphere."""
import numpy as np
from scipy import special

OBS = np.array([-0.534, -0.523, -0.644])     # observation direction of the paper's sphere figure


def pi_tau(mu, nmax):
    """Angular functions pi_n = P_n^1 / sin(theta), tau_n = dP_n^1 / dtheta (n = 1..nmax)."""
    pi = np.zeros((nmax + 1,) + np.shape(mu))
    tau = np.zeros_like(pi)
    pi[1] = 1.0
    tau[1] = mu
    for n in range(2, nmax + 1):
        pi[n] = (2 * n - 1) / (n - 1) * mu * pi[n - 1] - n / (n - 1) * pi[n - 2]
        tau[n] = n * mu * pi[n] - (n + 1) * pi[n - 1]
    return pi, tau


def surface_H(x, theta, phi, scattered=True):
    """Tangential H (theta, phi components) on the unit sphere at ka = x for E_i = x e^{ikz} (eta = 1)."""
    nmax = int(x + 4 * x ** (1 / 3) + 6)
    pi, tau = pi_tau(np.cos(theta), nmax)
    Ht = np.zeros(np.shape(theta), dtype=complex)
    Hp = np.zeros_like(Ht)
    for n in range(1, nmax + 1):
        jn, jd = special.spherical_jn(n, x), special.spherical_jn(n, x, derivative=True)
        yn, yd = special.spherical_yn(n, x), special.spherical_yn(n, x, derivative=True)
        hn, hd = jn + 1j * yn, jd + 1j * yd
        psi, dpsi = x * jn, jn + x * jd
        xi, dxi = x * hn, hn + x * hd
        a, b = (dpsi / dxi, psi / xi) if scattered else (0.0, 0.0)
        En = 1j ** n * (2 * n + 1) / (n * (n + 1))
        radial_j = jn - a * hn
        radial_n = 1j * (b * dxi - dpsi) / x
        Ht += En * np.sin(phi) * (pi[n] * radial_j + tau[n] * radial_n)
        Hp += En * np.cos(phi) * (tau[n] * radial_j + pi[n] * radial_n)
    return Ht, Hp


def frames(p):
    r = np.linalg.norm(p, axis=-1)
    th = np.arccos(np.clip(p[..., 2] / r, -1, 1))
    ph = np.arctan2(p[..., 1], p[..., 0])
    et = np.stack([np.cos(th) * np.cos(ph), np.cos(th) * np.sin(ph), -np.sin(th)], -1)
    ep = np.stack([-np.sin(ph), np.cos(ph), np.zeros_like(ph)], -1)
    return th, ph, et, ep


def points():
    rng = np.random.default_rng(2312063677)
    q = rng.standard_normal((8, 3))
    p = np.vstack([OBS, q])
    return p / np.linalg.norm(p, axis=1, keepdims=True)


def mie_current(p, t, t0=8.0, sigma=2.0, dw=0.005, wmax=7.0):
    """J(p, t) = n x H_total for the pulse exp(-((t - z - t0)/sigma)^2), by Fourier synthesis."""
    th, ph, et, ep = frames(p)
    w = (np.arange(int(wmax / dw)) + 0.5) * dw
    G = sigma * np.sqrt(np.pi) * np.exp(-(w * sigma) ** 2 / 4) * np.exp(1j * w * t0)
    J = np.zeros((len(t), len(p), 3))
    for wk, gk in zip(w, G):
        Ht, Hp = surface_H(wk, th, ph)
        Jw = Ht[:, None] * ep - Hp[:, None] * et           # r x (Ht t + Hp p) = Ht p - Hp t
        J += (gk * dw / np.pi * np.exp(-1j * wk * t)[:, None, None] * Jw[None]).real
    return J


def current_at(ops_topo, j, p):
    """sum_m j_m(t_n) f_m(q), q = the radial ray's hit on the mesh (j: nt x ne)."""
    V, F = ops_topo.V, ops_topo.F
    out = np.zeros((j.shape[0], len(p), 3))
    for i, d in enumerate(p):
        hit = None
        for c, (a, b, e) in enumerate(F):
            v0, v1, v2 = V[a], V[b], V[e]
            n = np.cross(v1 - v0, v2 - v0)
            den = n @ d
            if den <= 0:
                continue
            q = (n @ v0) / den * d
            l1 = np.cross(v2 - v1, q - v1) @ n
            l2 = np.cross(v0 - v2, q - v2) @ n
            l3 = np.cross(v1 - v0, q - v0) @ n
            if min(l1, l2, l3) >= -1e-12:
                hit = (c, q)
                break
        assert hit is not None
        c, q = hit
        for k in range(3):
            m = ops_topo.tedge[c, k]
            out[:, i, :] += j[:, m, None] * ops_topo.rwg(m, c, q[None])[0][None, :]
    return out
