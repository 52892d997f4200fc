"""Oracle pins: quasi-Helmholtz projectors (Sec. II-D) and the temporal basis (Sec. IV-A)."""
import json
import os

import numpy as np
import pytest

from oracle import cquad

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_facts.json")))


def _cholesky_projector(B):
    """B L^+ B^T through a Cholesky solve of L + 1 1^T / n (valid on zero-mean right-hand sides)."""
    L = B.T @ B
    n = L.shape[0]
    C = np.linalg.cholesky(L + np.ones((n, n)) / n)
    X = np.linalg.solve(C.T, np.linalg.solve(C, B.T))
    return B @ X


@pytest.mark.parametrize("which", ["sphere", "torus"])
def test_projector_algebra(which, ico1_fm, torus_fm):
    fm = ico1_fm if which == "sphere" else torus_fm
    t = fm.ops.topo
    I = np.eye(t.ne)
    PS, PL = fm.PS, fm.PPL
    PH = I - PS - PL
    for P in (PS, PL, PH):
        assert np.max(np.abs(P @ P - P)) < 1e-12
        assert np.max(np.abs(P - P.T)) < 1e-12
    assert np.max(np.abs(PS @ PL)) < 1e-12
    assert abs(np.trace(PS) - (t.nc - 1)) < 1e-9
    assert abs(np.trace(PL) - (t.nv - 1)) < 1e-9
    assert abs(np.trace(PH) - 2 * t.genus) < 1e-9
    # independent route to the pseudo-inverse
    assert np.max(np.abs(_cholesky_projector(fm.ops.Sig) - PS)) < 1e-11
    assert np.max(np.abs(_cholesky_projector(fm.ops.Lam) - PL)) < 1e-11
    # P^{Lambda H} Z^h = Z^h P^{Lambda H} = 0 structurally (Sec. III-B): H_k only sees stars
    H = fm.ops.H
    assert np.max(np.abs(np.einsum("ab,kbc->kac", fm.PLH, H))) < 1e-12 * np.max(np.abs(H))
    assert np.max(np.abs(fm.PPSH @ fm.ops.Zh)) < 1e-12 * np.max(np.abs(fm.ops.Zh))


def test_time_basis_closed_forms():
    L = cquad.lib()
    dt = 0.37
    for t, v in zip(GOLD["h0"]["t"], GOLD["h0"]["value"]):
        assert abs(L.oq_h0(t * dt, dt) - v) < 1e-15
    for t, v in zip(GOLD["q0"]["t"], GOLD["q0"]["value"]):
        assert abs(L.oq_q0(t * dt, dt) - v) < 1e-15
    grid = np.linspace(-3.0, 6.0, 901) * dt + 1e-9
    # partition of unity: sum_i h_i = 1 and sum_i q_i = 1
    sh = sum(np.array([L.oq_h0(x - i * dt, dt) for x in grid]) for i in range(-5, 10))
    sq = sum(np.array([L.oq_q0(x - i * dt, dt) for x in grid]) for i in range(-5, 10))
    assert np.max(np.abs(sh - 1.0)) < 1e-13 and np.max(np.abs(sq - 1.0)) < 1e-13
    # compatibility q_i' = (h_i - h_{i+1}) / dt (Sec. IV-B remark), by central differences
    eps = 1e-7 * dt
    for x in grid[::7]:
        dq = (L.oq_q0(x + eps, dt) - L.oq_q0(x - eps, dt)) / (2 * eps)
        assert abs(dq - (L.oq_h0(x, dt) - L.oq_h0(x - dt, dt)) / dt) < 1e-5 / dt
        dh = (L.oq_h0(x + eps, dt) - L.oq_h0(x - eps, dt)) / (2 * eps)
        assert abs(dh - L.oq_h0dot(x, dt)) < 1e-5 / dt
