"""Marching-on-in-time of the oracle (Sec. IV-B), three independent associations.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

  march_factored: per step, the retarded sums are formed from the shells S_k, H_k, MM_k,
      the projectors and L1, L2 (the equation of Sec. IV-A before the blocks are
      multiplied out); y_n is the solution of T_0 y_n = (known terms) by an FP64 LU
      with partial pivoting (numpy.linalg / LAPACK).
  march_dense:    y_n = T_0^{-1}(r_n - sum_{k>=1} T_k y_{n-k})  with the dense T_k (Sec. IV-B).
  block_solve:    the whole lower block-triangular system (Eq. dis_TD_CFIE) as one dense
                  linear system (brute force, tiny cases only).
Convention y_i = 0 for i <= 0 (causality, Sec. II-A).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .formulation import Formulation


def march_factored(fm: Formulation, r: np.ndarray) -> np.ndarray:
    """r: (Nt, ne, R) right-hand sides r_1..r_Nt.  Returns y (Nt, ne, R)."""
    o = fm.ops
    Nt, ne, R = r.shape
    K, dtt, a = o.K, fm.dtt, o.alpha
    left = dtt * fm.PLH + fm.PS
    A0 = 0.5 * o.G + o.MM[0]
    T0 = fm.L1 @ (left @ o.S[0] @ fm.J + o.H[0]) + a * fm.L2 @ (A0 @ fm.J)
    lu = sla.lu_factor(T0)
    y = np.zeros((Nt, ne, R))
    j = np.zeros((Nt, ne, R))
    for n in range(Nt):
        yprev = y[n - 1] if n >= 1 else np.zeros((ne, R))
        c = -fm.PS @ yprev / dtt
        es = o.S[0] @ c
        eh = np.zeros((ne, R))
        mm = A0 @ c
        for k in range(1, K):
            if n - k < 0:
                break
            es += o.S[k] @ j[n - k]
            eh += o.H[k] @ y[n - k]
            mm += o.MM[k] @ j[n - k]
        b = r[n] - fm.L1 @ (left @ es + eh) - a * fm.L2 @ mm
        y[n] = sla.lu_solve(lu, b)
        j[n] = fm.PLH @ y[n] + fm.PS @ (y[n] - yprev) / dtt
    return y


def march_dense(T: np.ndarray, r: np.ndarray) -> np.ndarray:
    """Direct MOT recurrence with the dense blocks T (K, ne, ne)."""
    K = T.shape[0]
    Nt, ne, R = r.shape
    lu = sla.lu_factor(T[0])
    y = np.zeros((Nt, ne, R))
    for n in range(Nt):
        b = r[n].copy()
        for k in range(1, K):
            if n - k < 0:
                break
            b -= T[k] @ y[n - k]
        y[n] = sla.lu_solve(lu, b)
    return y


def block_solve(T: np.ndarray, r: np.ndarray) -> np.ndarray:
    """Solve the (Nt ne) x (Nt ne) lower block-Toeplitz system in one dense solve."""
    K = T.shape[0]
    Nt, ne, R = r.shape
    A = np.zeros((Nt * ne, Nt * ne))
    for i in range(Nt):
        for k in range(min(K, i + 1)):
            A[i * ne:(i + 1) * ne, (i - k) * ne:(i - k + 1) * ne] = T[k]
    y = np.linalg.solve(A, r.reshape(Nt * ne, R))
    return y.reshape(Nt, ne, R)


def companion_spectral_radius(T: np.ndarray) -> float:
    """Largest |lambda| of the polynomial eigenproblem sum_k T_k lambda^{-k} x = 0 (Sec. V),
    via the block companion matrix of the recurrence y_n = -T_0^{-1} sum_{k>=1} T_k y_{n-k}."""
    K, ne, _ = T.shape
    if K == 1:
        return 0.0
    T0inv = np.linalg.inv(T[0])
    C = np.zeros(((K - 1) * ne, (K - 1) * ne))
    for k in range(1, K):
        C[:ne, (k - 1) * ne:k * ne] = -T0inv @ T[k]
    for k in range(1, K - 1):
        C[k * ne:(k + 1) * ne, (k - 1) * ne:k * ne] = np.eye(ne)
    return float(np.max(np.abs(np.linalg.eigvals(C))))
