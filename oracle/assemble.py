"""Space-time matrices of the oracle (Sec. II-A..C and IV-A), natural units c = eta = 1.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Retarded matrices per time lag k (Dirac testing at t_n of a basis centred at t_{n-k}); the time
basis is the paper's hat / C1-quadratic pair (time_order 1) or the shifted quadratic Lagrange
pair of the remark closing Sec. IV-B (time_order 2, see quad.c):
  S_k[m,n]   = -int int f_m(x).f_n(y) hdot_0(k dt - R) / (4 pi R)           (T^s, Sec. II-A)
  Phi_k[c,c'] = -T0 / (A_c A_c') int_c int_c' q_0(k dt - R) / (4 pi R)        (T^h on q-basis)
  H_k = Sigma Phi_k Sigma^T                                                  (charges div f = Sigma/A)
  MM_k[m,n]  = int int g_m(x).[R-hat x f_n(y)] (h_0/(4 pi R^2) + hdot_0/(4 pi R))  (K, Sec. II-A)
Static (Yukawa, kappa = 1/(c dt), Sec. II-B, II-C):
  G[m,n]  = <n x g_m, f_n>
  Zs[m,n] = -kappa int int g_m.g_n exp(-kappa R)/(4 pi R)
  Zh      = Lambda Psi Lambda^T,  Psi[v,v'] = -(1/kappa) int int rho_v rho_v' exp(-kappa R)/(4 pi R)
  M[m,n]  = int int g_m.[R-hat x f_n] (1 + kappa R) exp(-kappa R)/(4 pi R^2)
"""
from __future__ import annotations

import numpy as np

from . import cquad
from .bc import BarycentricBC
from .cquad import D, I, P
from .topology import Topology, n_lags

# 3-point degree-2 rule (barycentric), exact for the quadratic integrand of G
_R3_L = np.array([[2 / 3, 1 / 6, 1 / 6], [1 / 6, 2 / 3, 1 / 6], [1 / 6, 1 / 6, 2 / 3]])


class Operators:
    """All matrices of one mesh and time step (dense, FP64)."""

    def __init__(self, V, F, dt: float, alpha: float = 1.0, K: int | None = None, with_static: bool = True,
                 time_order: int = 1):
        self.time_order = int(time_order)      # 1: hat / C1-quadratic pair; 2: shifted quadratic Lagrange
        self.topo = topo = Topology(V, F)
        self.bc = bc = BarycentricBC(topo)
        self.dt = float(dt)
        self.alpha = float(alpha)
        self.T0 = topo.D                       # T0 = D / c
        self.dtt = self.dt / self.T0           # Delta-tilde t (Sec. III-A)
        self.kappa = 1.0 / self.dt             # kappa = 1/(c dt) (Sec. II-B)
        self.K = n_lags(topo.D, dt, self.time_order) if K is None else int(K)
        self.Lam = topo.Lambda().astype(np.float64)
        self.Sig = topo.Sigma().astype(np.float64)
        self._retarded()
        if with_static:
            self._static()

    # ------------------------------------------------------------------
    def _retarded(self):
        t, b = self.topo, self.bc
        ne, nc, K = t.ne, t.nc, self.K
        L = cquad.lib()
        S = np.zeros((K, ne, ne))
        Phi = np.zeros((K, nc, nc))
        MM = np.zeros((K, ne, ne))
        cquad.set_time_order(self.time_order)
        try:
            L.oq_retarded_efie(P(t.V), I(nc), P(t.F), I(ne), P(t.tedge), P(t.tsign), D(self.dt), I(K), D(self.T0),
                               D(t.D), P(S), P(Phi))
            L.oq_retarded_mfie(P(t.V), I(nc), P(t.F), I(ne), P(t.tedge), P(t.tsign),
                               P(b.fV), I(b.nf), P(b.fF), P(b.fparent), P(b.bc_ptr), P(b.bc_fn), P(b.bc_phi),
                               D(self.dt), I(K), D(t.D), P(MM))
        finally:
            cquad.set_time_order(1)
        self.S, self.Phi, self.MM = S, Phi, MM
        self.H = np.stack([self.Sig @ Phi[k] @ self.Sig.T for k in range(K)])

    def _static(self):
        t, b = self.topo, self.bc
        ne, nv = t.ne, t.nv
        L = cquad.lib()
        Zs = np.zeros((ne, ne))
        Psi = np.zeros((nv, nv))
        L.oq_static_efie(P(t.F), P(b.fV), I(b.nf), P(b.fF), P(b.fparent), P(b.fvert), P(t.valence), I(nv),
                         P(b.bc_ptr), P(b.bc_fn), P(b.bc_phi), I(ne), D(self.kappa), P(Zs), P(Psi))
        M = np.zeros((ne, ne))
        L.oq_static_mfie(P(t.V), I(t.nc), P(t.F), I(ne), P(t.tedge), P(t.tsign),
                         P(b.fV), I(b.nf), P(b.fF), P(b.fparent), P(b.bc_ptr), P(b.bc_fn), P(b.bc_phi),
                         D(self.kappa), P(M))
        self.Zs, self.Psi, self.M = Zs, Psi, M
        self.Zh = self.Lam @ Psi @ self.Lam.T
        self.G = gram(t, b)


def gram(t: Topology, b: BarycentricBC) -> np.ndarray:
    """G[m,n] = int (n x g_m) . f_n over the fine triangles (degree-2 rule, exact)."""
    G = np.zeros((t.ne, t.ne))
    for ft in range(b.nf):
        c = int(b.fparent[ft])
        w = b.fV[b.fF[ft]]
        pts = _R3_L @ w
        wts = np.full(3, b.farea[ft] / 3.0)
        nrm = t.normal[c]
        for e in range(b.bc_ptr[ft], b.bc_ptr[ft + 1]):
            m = int(b.bc_fn[e])
            g = np.zeros((3, 3))
            for j in range(3):
                g += b.bc_phi[e, j] * (pts - w[j]) / (2.0 * b.farea[ft])
            ng = np.cross(nrm[None, :], g)
            for j in range(3):
                n = int(t.tedge[c, j])
                f = t.tsign[c, j] * (pts - t.V[t.F[c, j]]) / (2.0 * t.area[c])
                G[m, n] += np.sum(wts * np.einsum("ij,ij->i", ng, f))
    return G
