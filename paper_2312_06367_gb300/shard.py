"""Row-sharded MOT march over several ranks: the partition and exchange logic (host side).

One large scatterer whose blocks exceed one device is split by rows: rank p holds rows
[lo_p, hi_p) of every T_k (k = 1 .. K-1), of the right-hand-side operator and of T_0^-1, with the
row boundaries on 128-row tiles so that each rank's history sum is whole tensor-core row tiles.
Per step n (Sec. IV-B):
    b_n[rows_p] = r_n[rows_p] - sum_{k>=1} T_k[rows_p, :] y_{n-k}      (local: no communication)
    b_n         = all-gather of the row blocks
    y_n[rows_p] = T_0^-1[rows_p, :] b_n                                 (local)
    y_n         = all-gather of the row blocks (every rank keeps the whole ring of y)
Two all-gathers of N x R values per step; the history sum, which streams (K - 1) N^2 / P entries
per rank, needs none.  The local products are injected (`matvec`), so the same exchange runs with
the library's kernels on devices and with plain numpy on CPU ranks (how it is tested here: one
GPU per call in this build, so the multi-device form is not measured on hardware).
"""
from __future__ import annotations

import numpy as np


def row_ranges(n: int, world: int, tile: int = 128):
    """Contiguous row ranges, one per rank, on tile boundaries, balanced to within one tile."""
    tiles = (n + tile - 1) // tile
    out = []
    for p in range(world):
        a = (p * tiles) // world * tile
        b = ((p + 1) * tiles) // world * tile
        out.append((min(a, n), min(b, n)))
    return out


def rowwise_matvec(M: np.ndarray, x: np.ndarray) -> np.ndarray:
    """M (rows, n) times x (n, R) with a fixed per-row summation order (no BLAS blocking), so a
    row's result does not depend on which other rows are computed with it."""
    return np.einsum("ij,jr->ir", M, x, optimize=False)


class ShardedMarch:
    """The rank-local state of the row-sharded march.

    T_rows:   (K, rows, n) rows [lo, hi) of T_0 .. T_{K-1} (T_0's rows are not used by the step)
    T0inv_rows: (rows, n) rows [lo, hi) of T_0^-1
    allgather: callable(local (rows, R) array) -> full (n, R) array in rank order
    """

    def __init__(self, T_rows, T0inv_rows, lo: int, hi: int, n: int, R: int, allgather, matvec=rowwise_matvec):
        self.T, self.T0inv = T_rows, T0inv_rows
        self.lo, self.hi, self.n, self.R = lo, hi, n, R
        self.K = T_rows.shape[0]
        self.allgather = allgather
        self.mv = matvec
        self.ring = [np.zeros((n, R)) for _ in range(self.K - 1)]   # y_{n-1} .. y_{n-K+1}
        self.step_no = 0

    def step(self, r_rows: np.ndarray) -> np.ndarray:
        """r_rows: (rows, R) right-hand side rows of step n.  Returns the whole y_n (n, R)."""
        self.step_no += 1
        b = np.array(r_rows, dtype=np.float64, copy=True)
        for k in range(1, self.K):
            if self.step_no - k < 1:
                break
            b -= self.mv(self.T[k], self.ring[(self.step_no - k) % (self.K - 1)])
        b_full = self.allgather(b)
        y_rows = self.mv(self.T0inv, b_full)
        y = self.allgather(y_rows)
        self.ring[self.step_no % (self.K - 1)] = y
        return y
