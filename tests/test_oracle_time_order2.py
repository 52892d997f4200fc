"""The higher-order temporal pair of the remark closing Sec. IV-B: shifted quadratic Lagrange
interpolators h_i for the solenoidal part and q_i with q_i' = (h_i - h_{i+1}) / dt for the
irrotational part (oracle/quad.c, time order 2).

* The pair itself: h_0 interpolates (h_0(j dt) = delta_j0), the shifted family reproduces 1, t and
  t^2 exactly, q_0' = (h_0(t) - h_0(t - dt)) / dt, the q_i sum to 1, and both vanish outside
  [-dt, 2 dt] and [-dt, 3 dt].
* The march with it: on the 80-triangle sphere it stays stable (the polynomial eigenvalues stay
  inside the unit circle, spectral radius as for the hat pair) and at dt 0.4 and 0.2 it is more
  than twice as accurate as the hat pair against a dt = 0.05 march.
"""
import numpy as np
import pytest

from oracle import cquad
from synth import excitation, meshes


@pytest.fixture()
def order2():
    L = cquad.lib()
    cquad.set_time_order(2)
    yield L
    cquad.set_time_order(1)


def test_quadratic_pair_closed_form_properties(order2):
    L = order2
    h = lambda t: L.oq_h0(float(t), 1.0)
    q = lambda t: L.oq_q0(float(t), 1.0)
    assert [h(j) for j in range(-3, 5)] == [0, 0, 0, 1, 0, 0, 0, 0]
    ts = np.linspace(-0.97, 3.93, 211)
    for p in range(3):                        # reproduces 1, t, t^2
        got = np.array([sum((i ** p) * h(t - i) for i in range(-4, 8)) for t in ts])
        assert np.allclose(got, ts ** p, atol=1e-12)
    assert np.allclose([sum(q(t - i) for i in range(-5, 9)) for t in ts], 1.0, atol=1e-12)
    eps = 1e-6
    for t in ts:
        dq = (q(t + eps) - q(t - eps)) / (2 * eps)
        assert abs(dq - (h(t) - h(t - 1.0))) < 1e-6
    out = [-1.5, -1.0, 2.0, 2.5]
    assert all(h(t) == 0.0 for t in out)
    assert all(q(t) == 0.0 for t in (-1.5, -1.0, 3.0, 3.5))
    assert max(abs(q(t)) for t in np.linspace(2.01, 2.99, 50)) > 0.01      # q_0 reaches 3 dt


def _march(dt, order, Tend=16.0):
    from oracle import comparators, mot, rhs
    from oracle.assemble import Operators
    from oracle.formulation import Formulation
    V, F = meshes.icosphere(1)
    pw = excitation.single(t0=6.0, sigma=1.5)
    ops = Operators(V, F, dt=dt, time_order=order)
    fm = Formulation(ops)
    nt = int(round(Tend / dt))
    e, h = rhs.incident_tests(ops, pw, dt * np.arange(1, nt + 1))
    j = fm.postprocess(mot.march_factored(fm, fm.rhs(e, h)))[..., 0]
    rho = np.abs(comparators.polynomial_eigenvalues(list(fm.T_stack()))).max()
    return j, ops.K, rho


def test_quadratic_pair_march_stable_and_more_accurate():
    ref, K_ref, rho_ref = _march(0.05, 2)
    assert K_ref == int(np.ceil(meshes_D() / 0.05 + 3.0)) and rho_ref < 1.0
    err = {}
    for dt in (0.4, 0.2):
        stride = int(round(dt / 0.05))
        r = ref[stride - 1::stride]
        for order in (1, 2):
            j, K, rho = _march(dt, order)
            n = min(len(j), len(r))
            err[dt, order] = np.linalg.norm(j[:n] - r[:n]) / np.linalg.norm(r[:n])
            assert rho < 1.0
    print("rel err vs dt 0.05 (order 2):", {k: f"{v:.2e}" for k, v in err.items()})
    for dt in (0.4, 0.2):
        assert err[dt, 2] < 0.5 * err[dt, 1]
    assert err[0.2, 1] < err[0.4, 1] and err[0.2, 2] < err[0.4, 2]


def meshes_D():
    from oracle.topology import Topology
    V, F = meshes.icosphere(1)
    return Topology(V, F).D


@pytest.mark.parametrize("order", [1, 2])
def test_blocks_vanish_beyond_the_lag_count(order):
    """Assembled with two extra lags, the retarded blocks past K = ceil(D/dt + order + 1) are zero
    and the last one inside is not: the support of q_0 ends at (order + 1) dt."""
    from oracle.assemble import Operators
    from oracle.topology import Topology, n_lags
    V, F = meshes.icosphere(1)
    dt = 0.4
    K = n_lags(Topology(V, F).D, dt, order)
    ops = Operators(V, F, dt=dt, K=K + 2, with_static=False, time_order=order)
    for k in (K, K + 1):
        assert not ops.S[k].any() and not ops.MM[k].any() and not ops.Phi[k].any()
    assert ops.Phi[K - 1].any()
