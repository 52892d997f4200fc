"""Oracle pins: the inner polar rule against closed forms and an independent adaptive integration.

The paper states no quadrature; these pins fix the rule's accuracy independently of itself:
  * int_T 1/R dS: closed form for a flat triangle (edge-by-edge log/arctan formula);
  * d int_T 1/R^3 dS = signed solid angle (Van Oosterom-Strackee);
  * retarded kernels with temporal breakpoints: 1-D adaptive integration in the polar angle
    of the exact radial antiderivative int f(R) dR (scipy.integrate.quad);
  * refinement of the rule's orders changes the assembled matrices by < 1e-7 of their largest
    entry (measured: S 3e-11, Phi 4e-9, MM 5e-8 on the 80-triangle sphere).
"""
import numpy as np
import pytest
from scipy import integrate

from oracle import cquad

TRI = [np.array([0.0, 0.0, 0.0]), np.array([1.0, 0.1, 0.0]), np.array([0.2, 0.9, 0.0])]
POINTS = [
    [0.3, 0.3, 0.0], [0.3, 0.3, 0.2], [0.3, 0.3, -0.05], [1.5, 1.2, 0.4], [-0.4, 0.2, 0.01],
    [0.5, 0.05, 0.3], [3.0, -2.0, 1.0], [0.45, 0.5, 1e-3],
]


def potential_closed_form(x, v):
    n = np.cross(v[1] - v[0], v[2] - v[0])
    n /= np.linalg.norm(n)
    d = np.dot(x - v[0], n)
    rho = x - d * n
    ad = abs(d)
    total = 0.0
    for i in range(3):
        a, b = v[i], v[(i + 1) % 3]
        l = (b - a) / np.linalg.norm(b - a)
        u = np.cross(l, n)
        P0 = np.dot(a - rho, u)
        lp, lm = np.dot(b - rho, l), np.dot(a - rho, l)
        Rp, Rm = np.linalg.norm(x - b), np.linalg.norm(x - a)
        R02 = P0 * P0 + d * d
        if abs(P0) > 1e-15:
            total += P0 * np.log((Rp + lp) / (Rm + lm))
            total -= ad * (np.arctan(P0 * lp / (R02 + ad * Rp)) - np.arctan(P0 * lm / (R02 + ad * Rm)))
    return total


def solid_angle(x, v):
    a, b, c = (vi - x for vi in v)
    la, lb, lc = (np.linalg.norm(z) for z in (a, b, c))
    num = np.dot(a, np.cross(b, c))
    den = la * lb * lc + np.dot(a, b) * lc + np.dot(a, c) * lb + np.dot(b, c) * la
    return 2.0 * np.arctan2(num, den)


@pytest.mark.parametrize("x", POINTS)
def test_single_layer_closed_form(x):
    x = np.array(x)
    m0, _ = cquad.triangle_moments(x, *TRI, kind=1, coplanar=(x[2] == 0.0))
    ref = potential_closed_form(x, TRI)
    assert abs(m0 - ref) < 1e-9 * abs(ref)


@pytest.mark.parametrize("x", [p for p in POINTS if p[2] != 0.0])
def test_double_layer_solid_angle(x):
    x = np.array(x)
    m0, m1 = cquad.triangle_moments(x, *TRI, kind=3)
    n = np.array([0.0, 0.0, 1.0])
    # int (y - x).n / R^3 = -d int 1/R^3 = solid angle
    om = solid_angle(x, TRI)
    assert abs(np.dot(m1, n) - om) < 1e-8 * max(1.0, abs(om))
    assert abs(-x[2] * m0 - om) < 1e-8 * max(1.0, abs(om))


def _adaptive_retarded(x, v, f, brk):
    """int_T f(R)/R dS by polar angle theta (adaptive) of the exact radial integral int f(R) dR."""
    n = np.array([0.0, 0.0, 1.0])
    d = x[2]
    p = np.array([x[0], x[1], 0.0])
    total = 0.0
    for i in range(3):
        a, b = v[i], v[(i + 1) % 3]
        sgn = np.sign(np.dot(np.cross(a - p, b - p), n))
        if sgn == 0:
            continue
        ta = np.arctan2(*(a - p)[[1, 0]])
        tb = ta + np.arctan2(np.dot(np.cross(a - p, b - p), n), np.dot(a - p, b - p))
        e = b - a

        def rho_edge(th):
            w = np.array([np.cos(th), np.sin(th), 0.0])
            # p + s w on the line a + t e
            M = np.array([[w[0], -e[0]], [w[1], -e[1]]])
            s, _ = np.linalg.solve(M, (a - p)[:2])
            return s

        def inner(th):
            Re = np.sqrt(rho_edge(th) ** 2 + d * d)
            pts = [r for r in brk if abs(d) < r < Re]
            val, _ = integrate.quad(f, abs(d), Re, points=pts or None, limit=200, epsabs=1e-14, epsrel=1e-13)
            return val

        lo, hi = min(ta, tb), max(ta, tb)
        val, _ = integrate.quad(inner, lo, hi, limit=400, epsabs=1e-13, epsrel=1e-12)
        total += val if tb > ta else -val
    return total


@pytest.mark.parametrize("x", [[0.3, 0.3, 0.05], [1.2, 0.9, 0.3], [0.5, 0.4, 0.0]])
@pytest.mark.parametrize("kind", [4, 5])
def test_retarded_kernels_with_breakpoints(x, kind):
    x = np.array(x)
    dt = 0.11
    k = 5
    brk = [j * dt for j in range(1, 40)]
    L = cquad.lib()
    if kind == 4:
        f = lambda R: L.oq_q0(k * dt - R, dt)
    else:
        f = lambda R: L.oq_h0dot(k * dt - R, dt)
    m0, _ = cquad.triangle_moments(x, *TRI, kind=kind, p1=k * dt, p2=dt, brk=brk, coplanar=(x[2] == 0.0))
    ref = _adaptive_retarded(x, TRI, f, brk)
    assert abs(m0 - ref) < 1e-8 * max(1e-3, abs(ref)), (m0, ref)


# every vertex of TRI at least two longest edges (2.28) from the projection: the far form applies
FAR_POINTS = [[3.0, -2.0, 1.0], [4.0, 3.5, 0.4], [-3.0, 0.4, 0.8], [0.5, -3.2, 0.05], [3.5, 3.0, 0.3]]


@pytest.mark.parametrize("x", FAR_POINTS)
def test_far_rule_closed_forms(x):
    """The far-pair rule (angle over the triangle's own range, no signed cancellation)."""
    x = np.array(x)
    m0, _ = cquad.triangle_moments(x, *TRI, kind=1, coplanar=2)
    ref = potential_closed_form(x, TRI)
    assert abs(m0 - ref) < 1e-9 * abs(ref)
    m0, m1 = cquad.triangle_moments(x, *TRI, kind=3, coplanar=2)
    om = solid_angle(x, TRI)
    assert abs(m1[2] - om) < 1e-7 * abs(om)


@pytest.mark.parametrize("x", [[3.2, 2.9, 0.3], [-2.5, -1.5, 0.2], [1.0, 3.5, 0.6]])
@pytest.mark.parametrize("kind", [4, 5])
def test_far_rule_with_breakpoints(x, kind):
    x = np.array(x)
    dt = 0.11
    k = int(np.linalg.norm(x - np.array([0.4, 0.33, 0.0])) / dt) + 1
    brk = [j * dt for j in range(1, 80)]
    L = cquad.lib()
    f = (lambda R: L.oq_q0(k * dt - R, dt)) if kind == 4 else (lambda R: L.oq_h0dot(k * dt - R, dt))
    m0, _ = cquad.triangle_moments(x, *TRI, kind=kind, p1=k * dt, p2=dt, brk=brk, coplanar=2)
    ref = _adaptive_retarded(x, TRI, f, brk)
    assert abs(m0 - ref) < 1e-8 * max(1e-3, abs(ref)), (m0, ref)


def test_rule_refinement_changes_matrices_little():
    from oracle.assemble import Operators
    from synth import meshes
    V, F = meshes.icosphere(1)
    try:
        a = Operators(V, F, dt=0.4, with_static=False)
        cquad.set_rule(10, 8, 0.5)
        b = Operators(V, F, dt=0.4, with_static=False)
    finally:
        cquad.set_rule(cquad.NANG, cquad.NRAD, cquad.PIECE)
    for A, B in ((a.S, b.S), (a.Phi, b.Phi), (a.MM, b.MM)):
        assert np.max(np.abs(A - B)) < 1e-7 * np.max(np.abs(A))
