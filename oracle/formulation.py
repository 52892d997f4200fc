"""Quasi-Helmholtz projectors and the qHP TD-CFIE blocks of the oracle (Sec. II-D, III, IV-A).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

  P^Sigma = Sigma (Sigma^T Sigma)^+ Sigma^T,  P^{Lambda H} = I - P^Sigma          (Sec. II-D)
  PP^Lambda = Lambda (Lambda^T Lambda)^+ Lambda^T,  PP^{Sigma H} = I - PP^Lambda   (Sec. II-D)
  Z~ = (dtt PP^{SH} + PP^L) Zs (PP^{SH} + PP^L/dtt) + PP^L Zh PP^L / dtt            (Sec. III-B)
  X~ = (dtt PP^{SH} + PP^L)(G/2 - M)                                              (Sec. III-C)
  L1 = Z~ G^{-T},  L2 = X~ G^{-1}                                                  (Eq. qHP_TDCFIE)
Dense time blocks (Sec. IV-A, Eq. dis_TD_CFIE), reading: T_k couples y_{n-k} to the test at t_n:
  ZZ~_k = (dtt P^{LH} + P^S)[S_k P^{LH} + (S_k - S_{k-1}) P^S / dtt] + H_k
  XX~_k = (G/2 d_{k0} + MM_k)(P^{LH} + P^S/dtt) - (G/2 d_{k1} + MM_{k-1}) P^S / dtt
  T_k   = L1 ZZ~_k + alpha L2 XX~_k
These follow from y(t) = sum_i (h_i P^{LH} + q_i P^S) y_i (Eq. y_expansion), j = (P^{LH} +
T0 d/dt P^S) y (Eq. j) and q_i' = (h_i - h_{i+1})/dt, which give j(t) = sum_i h_i(t) j_i with
j_i = P^{LH} y_i + P^S (y_i - y_{i-1}) / dtt (Eq. post_processing).
"""
from __future__ import annotations

import numpy as np

from .assemble import Operators


def pinv_projector(B: np.ndarray) -> np.ndarray:
    """B (B^T B)^+ B^T with the Moore-Penrose pseudo-inverse (numpy SVD)."""
    return B @ np.linalg.pinv(B.T @ B) @ B.T


class Formulation:
    def __init__(self, ops: Operators):
        self.ops = ops
        ne = ops.topo.ne
        I = np.eye(ne)
        self.PS = pinv_projector(ops.Sig)          # P^Sigma
        self.PLH = I - self.PS                     # P^{Lambda H}
        self.PPL = pinv_projector(ops.Lam)         # PP^Lambda (BC stars; also RWG local loops)
        self.PPSH = I - self.PPL                   # PP^{Sigma H}
        dtt = ops.dtt
        self.dtt = dtt
        if hasattr(ops, "Zs"):
            left = dtt * self.PPSH + self.PPL
            self.Zt = left @ ops.Zs @ (self.PPSH + self.PPL / dtt) + self.PPL @ ops.Zh @ self.PPL / dtt
            self.Xt = left @ (0.5 * ops.G - ops.M)
            Ginv = np.linalg.inv(ops.G)
            self.L1 = self.Zt @ Ginv.T
            self.L2 = self.Xt @ Ginv
        self.J = self.PLH + self.PS / dtt          # j_n = J y_n - P^S y_{n-1} / dtt

    # --------------------------------------------------------------
    def ZZt(self, k: int) -> np.ndarray:
        o = self.ops
        Sk = o.S[k] if k < o.K else 0.0 * o.S[0]
        Skm = o.S[k - 1] if 1 <= k <= o.K else 0.0 * o.S[0]
        Hk = o.H[k] if k < o.K else 0.0 * o.H[0]
        return (self.dtt * self.PLH + self.PS) @ (Sk @ self.PLH + (Sk - Skm) @ self.PS / self.dtt) + Hk

    def XXt(self, k: int) -> np.ndarray:
        o = self.ops
        z = 0.0 * o.MM[0]
        A = (0.5 * o.G if k == 0 else z) + (o.MM[k] if k < o.K else z)
        B = (0.5 * o.G if k == 1 else z) + (o.MM[k - 1] if 1 <= k <= o.K else z)
        return A @ (self.PLH + self.PS / self.dtt) - B @ self.PS / self.dtt

    def T(self, k: int) -> np.ndarray:
        return self.L1 @ self.ZZt(k) + self.ops.alpha * self.L2 @ self.XXt(k)

    def T_stack(self) -> np.ndarray:
        return np.stack([self.T(k) for k in range(self.ops.K)])

    def rhs(self, e: np.ndarray, h: np.ndarray) -> np.ndarray:
        """r_n = -L1 (dtt P^{LH} + P^S) e_n + alpha L2 h_n  (Sec. IV-A).  e, h: (Nt, ne, R)."""
        et = np.einsum("ab,nbr->nar", self.dtt * self.PLH + self.PS, e)
        return -np.einsum("ab,nbr->nar", self.L1, et) + self.ops.alpha * np.einsum("ab,nbr->nar", self.L2, h)

    def postprocess(self, y: np.ndarray) -> np.ndarray:
        """j_i = P^{LH} y_i + P^S (y_i - y_{i-1}) / dtt with y_0 = 0 (Eq. post_processing)."""
        yprev = np.concatenate([np.zeros_like(y[:1]), y[:-1]], axis=0)
        return np.einsum("ab,nbr->nar", self.PLH, y) + np.einsum("ab,nbr->nar", self.PS, y - yprev) / self.dtt
