"""Oracle pins: topology, incidence matrices and BC functions (Sec. II-C, II-D)."""
import json
import os

import numpy as np
import pytest

from oracle.bc import BarycentricBC
from oracle.topology import Topology, n_lags
from synth import meshes

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_facts.json")))

MESHES = {
    "tetra": meshes.tetrahedron(),
    "octa": meshes.octahedron(),
    "ico0": meshes.icosahedron(),
    "ico1": meshes.icosphere(1),
    "torus8x4": meshes.torus(1.0, 0.4, 8, 4),
    "torus12x6": meshes.torus(1.0, 0.4, 12, 6),
    "ellipsoid": meshes.ellipsoid(2, (2.0, 1.0, 0.5)),
    "jitter": meshes.perturbed(*meshes.icosphere(1), 0.1, seed=7),
}


@pytest.mark.parametrize("name", list(MESHES))
def test_incidence_identities(name):
    t = Topology(*MESHES[name])
    L, S = t.Lambda(), t.Sigma()
    # Sigma^T Lambda = 0, bit-exact in integers (orientation pairing of Sec. II-D)
    assert np.array_equal(S.T @ L, np.zeros((t.nc, t.nv), dtype=np.int64))
    # each row: one +1 and one -1
    for M in (L, S):
        assert np.all(np.sort(M, axis=1)[:, [0, -1]] == np.array([-1, 1]))
        assert np.all(np.abs(M).sum(axis=1) == 2)
    # Euler / genus (Sec. II-D harmonic dimension 2 g for a closed surface)
    expect_g = 1 if name.startswith("torus") else 0
    assert t.genus == expect_g
    assert t.nv - t.ne + t.nc == 2 - 2 * expect_g
    # ranks: N_C - 1 and N_V - 1 (connected surface)
    assert np.linalg.matrix_rank(S.astype(float)) == t.nc - 1
    assert np.linalg.matrix_rank(L.astype(float)) == t.nv - 1


def test_paper_mesh_counts_are_consistent():
    for key in ("sphere_mesh", "torus_mesh"):
        m = GOLD[key]
        assert m["vertices"] - m["edges"] + m["triangles"] == 2 - 2 * m["genus"]
    assert GOLD["harmonic_dimension"]["torus"] == 2 * GOLD["torus_mesh"]["genus"]


def test_config_sizes():
    for lvl, (nv, ne, nc) in {2: (162, 480, 320), 4: (2562, 7680, 5120)}.items():
        t = Topology(*meshes.icosphere(lvl))
        assert (t.nv, t.ne, t.nc) == (nv, ne, nc)
    t = Topology(*meshes.torus(1.0, 0.4, 24, 12))
    assert (t.nv, t.ne, t.nc, t.genus) == (288, 864, 576, 1)
    V, F = meshes.ellipsoid(5)
    assert F.shape[0] == 8192 and V.shape[0] == 4098


@pytest.mark.parametrize("name", ["octa", "ico1", "torus8x4", "jitter"])
def test_rwg_flux_and_divergence(name):
    """f_m has unit flux c+ -> c- across its edge and div f = +-1/A (Sec. II-C, Fig. 1)."""
    t = Topology(*MESHES[name])
    for m in range(t.ne):
        a, b = t.V[t.E[m, 0]], t.V[t.E[m, 1]]
        mid = 0.5 * (a + b)
        cp, cm = t.cplus[m], t.cminus[m]
        # in-plane normal of the edge pointing out of c+
        nout = np.cross(b - a, t.normal[cp])
        nout /= np.linalg.norm(nout)
        centre = t.V[t.F[cp]].mean(axis=0)
        assert np.dot(centre - mid, nout) < 0  # points away from c+
        fn = t.rwg(m, cp, mid[None, :])[0]
        assert np.isclose(np.dot(fn, nout) * np.linalg.norm(b - a), GOLD["rwg_flux"]["flux_through_edge"])
        # continuity of the normal component across the edge
        fm = t.rwg(m, cm, mid[None, :])[0]
        nin = np.cross(b - a, t.normal[cm])      # c- runs b -> a, so this points into c-
        nin /= np.linalg.norm(nin)
        assert np.isclose(np.dot(fm, nin) * np.linalg.norm(b - a), 1.0)


def test_diameter_and_lags():
    t = Topology(*meshes.icosphere(2))
    assert abs(t.D - 2.0) < 1e-12
    assert n_lags(t.D, 0.2) == 12           # T_0..T_11: 11 history blocks
    assert n_lags(2.0, 0.05) == 42
    assert n_lags(2.8, 2.0) == 4


@pytest.mark.parametrize("name", ["octa", "ico1", "torus8x4", "jitter"])
def test_bc_charges(name):
    """Every fine triangle of D_{v+} carries charge +1/(2 N_v), of D_{v-} -1/(2 N_v), else 0."""
    t = Topology(*MESHES[name])
    b = BarycentricBC(t)
    Q = b.charges()
    expect = np.zeros_like(Q)
    for n in range(t.ne):
        vm, vp = t.E[n]
        for ft in range(b.nf):
            v = b.fvert[ft]
            if v == vp:
                expect[ft, n] = 1.0 / (2 * t.valence[v])
            elif v == vm:
                expect[ft, n] = -1.0 / (2 * t.valence[v])
    assert np.max(np.abs(Q - expect)) < 1e-14
    # BC loops (Sigma-bar gives loops in the BC basis, Sec. II-D) are divergence-free
    loops = Q @ t.Sigma().astype(float)
    assert np.max(np.abs(loops)) < 1e-14
    # support: D_{v+} union D_{v-}
    assert b.nf == 6 * t.nc


@pytest.mark.parametrize("name", ["octa", "ico1", "torus12x6"])
def test_bc_normal_flux_continuity(name):
    """The normal component of g_n is continuous across every interior fine edge."""
    t = Topology(*MESHES[name])
    b = BarycentricBC(t)
    edge_flux = {}
    for ft in range(b.nf):
        tri = b.fF[ft]
        for e in range(b.bc_ptr[ft], b.bc_ptr[ft + 1]):
            n = b.bc_fn[e]
            for j in range(3):
                key = (n, min(tri[(j + 1) % 3], tri[(j + 2) % 3]), max(tri[(j + 1) % 3], tri[(j + 2) % 3]))
                edge_flux[key] = edge_flux.get(key, 0.0) + b.bc_phi[e, j]
    assert max(abs(v) for v in edge_flux.values()) < 1e-14


def test_gram_pins(ico1_ops, torus_ops):
    for ops in (ico1_ops, torus_ops):
        G = ops.G
        assert np.all(np.diag(G) > 0)
        S, L = ops.Sig, ops.Lam
        # Sigma^T G Lambda = 0: n x (BC loop) is a gradient, RWG loops are div-free
        assert np.max(np.abs(S.T @ G @ L)) < 1e-13 * np.max(np.abs(G))
        P = np.eye(G.shape[0]) - S @ np.linalg.pinv(S.T @ S) @ S.T - L @ np.linalg.pinv(L.T @ L) @ L.T
        assert np.max(np.abs(S.T @ G @ P)) < 1e-13 * np.max(np.abs(G))
        assert np.linalg.cond(G) < 10.0


def test_gram_condition_bounded_under_refinement():
    from oracle.assemble import gram
    conds = []
    for lvl in (1, 2, 3):
        t = Topology(*meshes.icosphere(lvl))
        conds.append(np.linalg.cond(gram(t, BarycentricBC(t))))
    assert max(conds) < 10.0 and conds[-1] < 1.5 * conds[0]
