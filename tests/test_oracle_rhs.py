"""Pins of the oracle's plane-wave tests (right-hand side, Sec. II-C and IV-A), independent of its
quadrature and of its BC coefficient tables.

For a spatially uniform field the tests reduce to the integrals of the basis functions, and for a
normal-continuous tangential field f of compact support on a closed polyhedral surface,
int f dS = - int r div f dS (the surface divergence theorem applied to f x_i).  So:
  RWG f_m (div = +1/A on c+, -1/A on c-):  int f_m = c- - c+ (triangle centroids);
  BC g_m (div = Lambda_{m v} / (2 N_v) per fine triangle of the dual cell D_v, area-normalised):
      int g_m = - sum_v Lambda_{m v} sum_{t in D_v} centroid(t) / (2 N_v).
A pulse whose width is huge is uniform in space at t = t0."""
import numpy as np
import pytest

from oracle import rhs
from oracle.assemble import Operators
from synth import meshes


@pytest.fixture(scope="module", params=["icosphere1", "torus8x4"])
def ops(request):
    V, F = meshes.icosphere(1) if request.param == "icosphere1" else meshes.torus(1.0, 0.4, 8, 4)
    return Operators(V, F, dt=0.5)


def _uniform_pulse(k, p):
    return {"k": np.array([k]), "p": np.array([p]), "amp": np.ones(1), "t0": np.zeros(1), "sigma": np.full(1, 1e9)}


def test_e_tests_uniform_field(ops):
    t = ops.topo
    k = np.array([0.0, 0.6, 0.8])
    p = np.array([1.0, 0.0, 0.0])
    e, _ = rhs.incident_tests(ops, _uniform_pulse(k, p), np.array([0.0]))
    cen = t.V[t.F].mean(axis=1)
    ref = (cen[t.cminus] - cen[t.cplus]) @ p
    assert np.max(np.abs(e[0, :, 0] - ref)) < 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_h_tests_uniform_field(ops):
    t, b = ops.topo, ops.bc
    k = np.array([0.0, 0.6, 0.8])
    p = np.array([1.0, 0.0, 0.0])
    _, h = rhs.incident_tests(ops, _uniform_pulse(k, p), np.array([0.0]))
    fcen = b.fV[b.fF].mean(axis=1)
    # dual cell of coarse vertex v: the fine triangles whose coarse vertex is v
    cell_sum = np.zeros((t.nv, 3))
    np.add.at(cell_sum, b.fvert, fcen)
    cell = cell_sum / (2.0 * t.valence)[:, None]
    vminus, vplus = t.E[:, 0], t.E[:, 1]
    integral = -(cell[vplus] - cell[vminus])            # Lambda = +1 at v+, -1 at v-
    ref = integral @ np.cross(k, p)
    assert np.max(np.abs(h[0, :, 0] - ref)) < 1e-12 * max(1.0, np.max(np.abs(ref)))
