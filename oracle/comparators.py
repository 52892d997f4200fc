"""The paper's comparison formulations as test oracles (Sec. V): the standard TD-EFIE and the
mixed TD-MFIE, marched with the hat basis in time and Dirac testing on the same retarded matrices
as the qHP TD-CFIE (S_k, Phi_k, MM_k of oracle/assemble.py).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Mixed TD-MFIE (BC tests n x g_m, RWG trial, Sec. II-A and the MFIE row of Sec. II-C):
    (G/2 + MM) j = h   ->   sum_k MM'_k j_{n-k} = h_n,   MM'_k = MM_k + G/2 [k = 0].
Standard TD-EFIE (rotated RWG tests): (T^s + T^h) j = -e.  With j(t) = sum_i h_i(t) j_i, T^s gives
S_k.  T^h carries the time integral of h_i, the ramp r_0(t) = int h_0 = dt sum_{l >= 0} q_0(t - l dt)
(q_0' = (h_0 - h_1)/dt, Sec. IV-B), and Phi_k is built with q_0 and the factor -T0 (assemble.py), so
the T^h block at lag k is dtt sum_{l <= k} H_l with dtt = dt / T0 and H_l = Sigma Phi_l Sigma^T:
    Z_k = S_k + dtt sum_{l=0}^{min(k, K-1)} H_l,   sum_{k >= 0} Z_k j_{n-k} = -e_n.
Z_k stops changing for k >= K (Z_inf = dtt sum_l H_l), so the march keeps a running sum of the
currents older than K - 1 steps.  Differencing two consecutive steps gives the finite recurrence
    sum_{k=0}^{K} D_k j_{n-k} = -(e_n - e_{n-1}),   D_0 = Z_0,  D_k = S_k - S_{k-1} + dtt H_k,
whose polynomial sum_k D_k lambda^{-k} is what the stability test examines: sum_k D_k = Z_inf
vanishes on the loop currents (Sigma^T f = 0), the DC null space of the standard TD-EFIE.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def mfie_blocks(ops) -> list[np.ndarray]:
    """MM'_k, k = 0..K-1."""
    out = [m.copy() for m in ops.MM]
    out[0] = out[0] + 0.5 * ops.G
    return out


def march_mfie(ops, h: np.ndarray) -> np.ndarray:
    """Mixed TD-MFIE march: h (Nt, ne, R) tests -> j (Nt, ne, R)."""
    Z = mfie_blocks(ops)
    lu = sla.lu_factor(Z[0])
    Nt = h.shape[0]
    j = np.zeros_like(h)
    for n in range(Nt):
        b = h[n].copy()
        for k in range(1, len(Z)):
            if n - k < 0:
                break
            b -= Z[k] @ j[n - k]
        j[n] = sla.lu_solve(lu, b)
    return j


def efie_blocks(ops, dtt: float) -> tuple[list[np.ndarray], np.ndarray]:
    """Z_k for k = 0..K-1 and Z_inf."""
    K = ops.K
    Z, acc = [], np.zeros_like(ops.H[0])
    for k in range(K):
        acc = acc + ops.H[k]
        Z.append(ops.S[k] + dtt * acc)
    return Z, dtt * acc


def efie_difference_blocks(ops, dtt: float) -> list[np.ndarray]:
    """D_k, k = 0..K, of the differenced standard TD-EFIE recurrence."""
    K = ops.K
    S = list(ops.S) + [np.zeros_like(ops.S[0])]
    H = list(ops.H) + [np.zeros_like(ops.H[0])]
    return [S[0] + dtt * H[0]] + [S[k] - S[k - 1] + dtt * H[k] for k in range(1, K + 1)]


def march_efie(ops, dtt: float, e: np.ndarray) -> np.ndarray:
    """Standard TD-EFIE march: e (Nt, ne, R) tests -> j (Nt, ne, R)."""
    Z, Zinf = efie_blocks(ops, dtt)
    K = len(Z)
    lu = sla.lu_factor(Z[0])
    Nt = e.shape[0]
    j = np.zeros_like(e)
    old = np.zeros_like(e[0])           # sum of j_i for i <= n - K
    for n in range(Nt):
        if n - K >= 0:
            old += j[n - K]
        b = -e[n] - Zinf @ old
        for k in range(1, K):
            if n - k < 0:
                break
            b -= Z[k] @ j[n - k]
        j[n] = sla.lu_solve(lu, b)
    return j


def polynomial_eigenvalues(D: list[np.ndarray]) -> np.ndarray:
    """Eigenvalues lambda of sum_k D_k lambda^{-k} x = 0 (block companion matrix, dense eig)."""
    ne, K = D[0].shape[0], len(D) - 1
    D0i = np.linalg.inv(D[0])
    C = np.zeros((K * ne, K * ne))
    for k in range(1, K + 1):
        C[:ne, (k - 1) * ne:k * ne] = -D0i @ D[k]
    C[ne:, :-ne] = np.eye((K - 1) * ne)
    return np.linalg.eigvals(C)
