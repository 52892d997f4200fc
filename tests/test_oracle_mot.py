"""Oracle pins: the MOT recurrence, its stability and the static MFIE property (Sec. III-C, IV, V)."""
import numpy as np
import pytest

from oracle import mot, rhs
from oracle.assemble import Operators
from oracle.formulation import Formulation
from synth import excitation, meshes


def _run(V, F, dt, Nt, pw=None):
    ops = Operators(V, F, dt=dt)
    fm = Formulation(ops)
    T = fm.T_stack()
    pw = pw or excitation.single(t0=3.0, sigma=1.0)
    e, h = rhs.incident_tests(ops, pw, dt * np.arange(1, Nt + 1))
    return ops, fm, T, fm.rhs(e, h)


@pytest.mark.parametrize("mesh,dt", [("octa", 0.5), ("ico0", 0.4), ("tetra", 0.3)])
def test_march_equals_block_solve(mesh, dt):
    """Marching (Sec. IV-B) solves the lower block-Toeplitz system (Eq. dis_TD_CFIE) exactly."""
    V, F = {"octa": meshes.octahedron, "ico0": meshes.icosahedron, "tetra": meshes.tetrahedron}[mesh]()
    pw = excitation.random_batch(2, seed=5, t0=2.0, sigma=0.7)
    ops, fm, T, r = _run(V, F, dt, 14, pw)
    yb = mot.block_solve(T, r)
    yd = mot.march_dense(T, r)
    yf = mot.march_factored(fm, r)
    s = np.linalg.norm(yb)
    assert np.linalg.norm(yd - yb) < 1e-12 * s
    assert np.linalg.norm(yf - yb) < 1e-12 * s


def test_dense_blocks_vanish_beyond_K(ico1_fm):
    """T_k = 0 once (k - 2) dt >= D: the retarded supports end (temporal basis supports)."""
    o = ico1_fm.ops
    assert np.max(np.abs(ico1_fm.T(o.K))) == 0.0
    assert np.max(np.abs(ico1_fm.T(o.K - 1))) > 0.0


def test_postprocess_definition(ico1_fm):
    """j_i = P^LH y_i + P^S (y_i - y_{i-1}) / dtt with y_0 = 0 (Eq. post_processing)."""
    rng = np.random.default_rng(0)
    y = rng.standard_normal((5, ico1_fm.ops.topo.ne, 2))
    j = ico1_fm.postprocess(y)
    fm = ico1_fm
    assert np.allclose(j[0], fm.PLH @ y[0] + fm.PS @ y[0] / fm.dtt)
    assert np.allclose(j[3], fm.PLH @ y[3] + fm.PS @ (y[3] - y[2]) / fm.dtt)


@pytest.mark.parametrize("dt", [0.2, 0.5, 2.0])
def test_sphere_spectrum_inside_unit_circle(dt):
    """qHP TD-CFIE spectrum strictly inside the unit circle on the sphere (Sec. V-A)."""
    ops = Operators(*meshes.icosphere(1), dt=dt)
    T = Formulation(ops).T_stack()
    assert mot.companion_spectral_radius(T) < 0.99


def test_torus_spectrum_inside_unit_circle(torus_fm):
    """Torus (genus 1): poles inside the circle at a moderate time step (Sec. V-B)."""
    assert mot.companion_spectral_radius(torus_fm.T_stack()) < 0.99


def test_sphere_late_time_decay_without_floor(ico1_fm):
    """The qHP current decays without a floor, far below 1e-100 in FP64 (Sec. V-A)."""
    o = ico1_fm.ops
    T = ico1_fm.T_stack()
    Nt = 1500
    e, h = rhs.incident_tests(o, excitation.single(t0=8.0, sigma=2.0), o.dt * np.arange(1, Nt + 1))
    y = mot.march_dense(T, ico1_fm.rhs(e, h))
    j = ico1_fm.postprocess(y)
    nrm = np.linalg.norm(j.reshape(Nt, -1), axis=1)
    assert nrm[30:60].max() > 0.1
    assert nrm[-1] < 1e-100
    # windowed maxima after the pulse are non-increasing
    w = nrm[100:].reshape(-1, 50).max(axis=1)
    assert np.all(w[1:] <= w[:-1] * (1 + 1e-12))


def test_static_mfie_property_sphere():
    """PP^SH (G/2 - M0) G^-1 (G/2 + M0) P^LH ~ 0 (Eq. property), to discretisation accuracy."""
    ops = Operators(*meshes.icosphere(1), dt=1e5)
    fm = Formulation(ops)
    A = (0.5 * ops.G - ops.M) @ np.linalg.inv(ops.G) @ (0.5 * ops.G + ops.M)
    assert np.linalg.norm(fm.PPSH @ A @ fm.PLH) < 1e-4 * np.linalg.norm(A)
    # the property is homogeneous in M (it fixes M's structure, not its scale or sign);
    # swapping the test and trial roles (M^T) breaks it by two orders of magnitude
    B = (0.5 * ops.G - ops.M.T) @ np.linalg.inv(ops.G) @ (0.5 * ops.G + ops.M.T)
    assert np.linalg.norm(fm.PPSH @ B @ fm.PLH) > 1e-3 * np.linalg.norm(B)


def test_t0_well_conditioned_across_dt():
    """cond(T_0) stays bounded as dt grows (no large-time-step breakdown, Sec. V)."""
    V, F = meshes.icosphere(1)
    conds = [np.linalg.cond(Formulation(Operators(V, F, dt=dt)).T(0)) for dt in (0.1, 1.0, 10.0, 100.0)]
    assert max(conds) < 10.0


def test_t0_block_scaling_large_dt():
    """Large-time-step balance of the combined operator (Sec. IV, the scaling table of Eq.
    qHP_TDCFIE): in the [Lambda, Sigma] bases of the tested (rows: PP^Lambda, PP^{Sigma H}) and the
    unknown (columns: P^{Lambda H}, P^Sigma) spaces of the sphere (no harmonic part), the
    (Lambda, Sigma) block of T_0 falls as dt^-1 and the two diagonal blocks stay O(1).  The remaining
    (Sigma, Lambda) block vanishes in the continuous setting by the static MFIE property; discretely
    it is dtt times the residual PP^{Sigma H} (G/2 - M) G^-1 (G/2 + MM_0) P^{Lambda H}, which is small
    and whose dt-growth is exactly that factor."""
    V, F = meshes.icosphere(1)
    dts = (10.0, 100.0, 1000.0)
    blocks = {}
    resid = []
    for dt in dts:
        ops = Operators(V, F, dt=dt)
        fm = Formulation(ops)
        T0 = fm.T(0)
        for rn, R in (("L", fm.PPL), ("S", fm.PPSH)):
            for cn, C in (("L", fm.PLH), ("S", fm.PS)):
                blocks.setdefault(rn + cn, []).append(np.linalg.norm(R @ T0 @ C))
        MM0 = ops.MM[0]
        res = fm.PPSH @ (0.5 * ops.G - ops.M) @ np.linalg.inv(ops.G) @ (0.5 * ops.G + MM0) @ fm.PLH
        resid.append(np.linalg.norm(res))
    slope = {k: np.polyfit(np.log(dts), np.log(v), 1)[0] for k, v in blocks.items()}
    assert abs(slope["LS"] + 1.0) < 0.3
    assert abs(slope["LL"]) < 0.3 and abs(slope["SS"]) < 0.3
    # (Sigma, Lambda): small against the diagonal blocks over the range, and dtt-proportional
    assert max(blocks["SL"]) < 0.05 * min(min(blocks["LL"]), min(blocks["SS"]))
    ratio = np.array(blocks["SL"][1:]) / np.array(dts[1:])     # once MM_0 has reached its static limit
    assert np.max(ratio) / np.min(ratio) < 1.1
    assert max(resid) < 1e-2 * np.linalg.norm(0.5 * Operators(V, F, dt=dts[0]).G)
