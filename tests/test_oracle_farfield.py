"""Oracle pins of the far-field evaluation and the large-time-step accuracy test (Sec. V: the
sphere marched with c dt / D ~ 5e4 and its far field at 3 Hz compared with the series solution).

* Radiation integrals at k = 0 against the closed form int_{c+-} f_m dS = +-(centroid - r+-)/2
  (the RWG function is linear on each triangle), for random currents.
* Loop currents (j = Lambda l, divergence-free) have no k = 0 radiation vector.
* The hat-basis spectrum of a sampled Gaussian against its analytic transform.
* The Rayleigh far field against the textbook small-sphere patterns |cos(theta) - 1/2| (E-plane)
  and |1 - cos(theta)/2| (H-plane).
* Physics: the oracle's qHP TD-CFIE march of the 320-triangle sphere at dt = 1e5 (the paper's
  0.333 ms, pulse w = 8e6 m, t0 = 80 ms in metres of light travel), far field at 3 Hz against the
  Rayleigh limit of the sphere (k a = 6.3e-8, where it equals the series to O((ka)^2)).
"""
import numpy as np
import pytest

from oracle import farfield
from oracle.topology import Topology
from synth import excitation, meshes

K3HZ = 2.0 * np.pi * 3.0 / 299792458.0     # 3 Hz as a wavenumber (1/m); dt = 1e5 m of light travel is 0.334 ms


def _dirs():
    out = []
    for phi in (0.0, np.pi / 2):
        for t in np.linspace(0.1, np.pi - 0.1, 9):
            out.append([np.sin(t) * np.cos(phi), np.sin(t) * np.sin(phi), np.cos(t)])
    return np.array(out)


def test_radiation_integrals_closed_form_at_k0():
    V, F = meshes.icosphere(1)
    t = Topology(V, F)
    got = farfield.radiation_integrals(t, np.array([[0.0, 0.0, 1.0]]), 0.0)[0].real
    cen = V[F].mean(axis=1)
    want = 0.5 * (cen[t.cplus] - V[t.ropp_plus]) + 0.5 * (V[t.ropp_minus] - cen[t.cminus])
    assert np.abs(got - want).max() < 1e-14


def test_loop_currents_do_not_radiate_at_k0():
    V, F = meshes.icosphere(2)
    t = Topology(V, F)
    rng = np.random.default_rng(3)
    j = t.Lambda() @ rng.standard_normal(t.nv)
    N = np.einsum("mx,m->x", farfield.radiation_integrals(t, np.array([[1.0, 0.0, 0.0]]), 0.0)[0], j)
    assert np.abs(N).max() < 1e-13 * np.abs(j).max()


def test_hat_spectrum_of_a_gaussian():
    dt, s, t0 = 0.01, 1.0, 6.0
    tt = dt * np.arange(1, 1400)
    j = np.exp(-((tt - t0) / s) ** 2)[:, None, None]
    for w in (0.3, 1.0, 2.5):
        got = farfield.current_spectrum(j, dt, w)[0, 0]
        want = s * np.sqrt(np.pi) * np.exp(-(0.5 * w * s) ** 2) * np.exp(-1j * w * t0)
        assert abs(got - want) < 1e-4 * abs(want)


def test_rayleigh_patterns():
    E0, khat = np.array([1.0, 0.0, 0.0]), np.array([0.0, 0.0, 1.0])
    th = np.linspace(0.05, np.pi - 0.05, 13)
    e_plane = np.stack([np.sin(th), 0 * th, np.cos(th)], axis=1)
    h_plane = np.stack([0 * th, np.sin(th), np.cos(th)], axis=1)
    Fe = np.linalg.norm(farfield.rayleigh_sphere(e_plane, 1e-3, 1.0, E0, khat), axis=1) / 1e-6
    Fh = np.linalg.norm(farfield.rayleigh_sphere(h_plane, 1e-3, 1.0, E0, khat), axis=1) / 1e-6
    assert np.allclose(Fe, np.abs(np.cos(th) - 0.5), atol=1e-12)
    assert np.allclose(Fh, np.abs(1.0 - 0.5 * np.cos(th)), atol=1e-12)


@pytest.fixture(scope="module")
def sphere_large_dt():
    from oracle import mot, rhs
    from oracle.assemble import Operators
    from oracle.formulation import Formulation
    V, F = meshes.icosphere(2)
    dt = 1e5
    ops = Operators(V, F, dt=dt)
    fm = Formulation(ops)
    pw = excitation.single(t0=2.4e7, sigma=2e6)
    nt = 360
    e, h = rhs.incident_tests(ops, pw, dt * np.arange(1, nt + 1))
    return ops, pw, dt, fm.postprocess(mot.march_factored(fm, fm.rhs(e, h)))


def test_far_field_at_3hz_after_large_dt_march(sphere_large_dt):
    ops, pw, dt, j = sphere_large_dt
    assert ops.K == 3
    d = _dirs()
    Fc = farfield.far_field(ops.topo, j, dt, K3HZ, d)[:, 0, :]
    Fr = farfield.rayleigh_sphere(d, K3HZ, 1.0, farfield.incident_amplitude(pw, 0, K3HZ), pw["k"][0])
    err = np.linalg.norm(Fc - Fr) / np.linalg.norm(Fr)
    ratio = np.linalg.norm(Fc, axis=1) / np.linalg.norm(Fr, axis=1)
    print(f"320 triangles, dt 1e5, 3 Hz: far field rel err vs Rayleigh {err:.3e}, |F| ratio {ratio.min():.4f}..{ratio.max():.4f}")
    assert err < 0.05
    # the march has finished: the current decayed with the pulse
    assert np.abs(j[-5:]).max() < 1e-10 * np.abs(j).max()
