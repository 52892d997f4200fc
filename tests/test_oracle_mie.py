"""Physics pin of the oracle: sphere surface currents against the Mie-series transient.

A perfectly conducting unit sphere lit by the x-polarised Gaussian pulse E = x exp(-((t - z - 8)/2)^2)
travelling along +z (the 480-edge sphere workload, dt 0.2, 300 steps).  The reference current
J = n x H on the sphere comes from the frequency-domain Mie series (vector spherical wave functions,
exp(-i w t) convention, PEC coefficients a_n = psi_n'/xi_n', b_n = psi_n/xi_n) synthesised over the
pulse spectrum.  The series itself is pinned first, independently of the MOT: its incident part
must rebuild the plane wave, its low-frequency limit must give the magnetostatic surface field of a
sphere (3/2 of the incident tangential H), and the synthesised incident field must be the pulse.

The MOT current at a point is sum_m j_m f_m(r) on the triangle met by the radial ray (RWG functions
as the paper normalises them).  The paper prints no tolerance; 320 triangles resolve the pulse's
spectrum (up to ka ~ 4) with about 7 edges per wavelength, and the bar is rel-L2 <= 0.15 over
time and points (the observation direction of the paper's sphere figure plus 8 seeded points)."""
import numpy as np
import pytest

from mie_series import current_at, frames, mie_current, points, surface_H
from synth import workloads


def test_incident_expansion_rebuilds_plane_wave():
    p = points()
    th, ph, et, ep = frames(p)
    for x in (0.3, 2.0, 6.0):
        Ht, Hp = surface_H(x, th, ph, scattered=False)
        Hinc = np.exp(1j * x * p[:, 2])[:, None] * np.array([0.0, 1.0, 0.0])      # y e^{ikz}
        assert np.allclose(Ht, np.einsum("ij,ij->i", Hinc, et), atol=1e-10)
        assert np.allclose(Hp, np.einsum("ij,ij->i", Hinc, ep), atol=1e-10)


def test_low_frequency_limit_is_magnetostatic():
    """ka -> 0: a PEC sphere in a uniform H0 has tangential surface field (3/2) H0_tan."""
    p = points()
    th, ph, et, ep = frames(p)
    Ht, Hp = surface_H(1e-4, th, ph)            # corrections are O(ka)
    y = np.array([0.0, 1.0, 0.0])
    assert np.max(np.abs(Ht - 1.5 * et @ y)) < 1e-3
    assert np.max(np.abs(Hp - 1.5 * ep @ y)) < 1e-3


def test_synthesised_incident_field_is_the_pulse():
    p = points()[:3]
    th, ph, et, ep = frames(p)
    t = np.linspace(0.0, 20.0, 41)
    w = (np.arange(1400) + 0.5) * 0.005
    G = 2.0 * np.sqrt(np.pi) * np.exp(-(w * 2.0) ** 2 / 4) * np.exp(1j * w * 8.0)
    Hth = np.zeros((len(t), len(p)))
    for wk, gk in zip(w, G):
        Ht, _ = surface_H(wk, th, ph, scattered=False)
        Hth += (gk * 0.005 / np.pi * np.exp(-1j * wk * t)[:, None] * Ht[None]).real
    ref = np.exp(-((t[:, None] - p[None, :, 2] - 8.0) / 2.0) ** 2) * et[None, :, 1]
    assert np.max(np.abs(Hth - ref)) < 1e-8


@pytest.mark.slow
def test_mot_sphere_currents_match_mie_transient():
    from oracle import mot, rhs
    from oracle.assemble import Operators
    from oracle.formulation import Formulation
    w = workloads.sphere480_fp64()
    ops = Operators(w["V"], w["F"], dt=w["dt"], alpha=w["alpha"])
    fm = Formulation(ops)
    t = w["dt"] * np.arange(1, w["Nt"] + 1)
    e, h = rhs.incident_tests(ops, w["pw"], t)
    y = mot.march_factored(fm, fm.rhs(e, h))
    j = fm.postprocess(y)[:, :, 0]
    p = points()
    J_mot = current_at(ops.topo, j, p)
    J_mie = mie_current(p, t)
    err = np.linalg.norm(J_mot - J_mie) / np.linalg.norm(J_mie)
    err_obs = np.linalg.norm(J_mot[:, 0] - J_mie[:, 0]) / np.linalg.norm(J_mie[:, 0])
    print(f"MOT vs Mie transient: rel-L2 {err:.3f} (observation point {err_obs:.3f})")
    assert err < 0.15
    # planted mistake: the post-processing with the loop/star projectors swapped must fail the pin
    yp = np.concatenate([np.zeros_like(y[:1]), y[:-1]], axis=0)
    bad = (np.einsum("ab,nbr->nar", fm.PS, y) + np.einsum("ab,nbr->nar", fm.PLH, y - yp) / fm.dtt)[:, :, 0]
    err_bad = np.linalg.norm(current_at(ops.topo, bad, p) - J_mie) / np.linalg.norm(J_mie)
    assert err_bad > 3 * 0.15
