"""C-ABI library on the host: loads, exports every declared symbol, and its host tables
(edges, c+/c-, BC coefficients) equal the oracle's bit for bit (integers) or to rounding."""
import os
import re

import numpy as np
import pytest

from synth import meshes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2312_06367_gb300 import _lib
    return _lib.load()


def test_exports_every_declared_symbol(lib):
    hdr = open(os.path.join(ROOT, "include", "tdcfie.h")).read()
    declared = set(re.findall(r"^\s*(?:const char\*|void|tdcfie_status)\s+(tdcfie_\w+)\s*\(", hdr, re.M))
    assert len(declared) >= 12
    for name in declared:
        assert hasattr(lib, name), name
    from paper_2312_06367_gb300 import _lib
    assert {s[0] for s in _lib.SIGNATURES} == declared


MESHES = {"ico1": meshes.icosphere(1), "torus8x4": meshes.torus(1.0, 0.4, 8, 4),
          "ellipsoid": meshes.ellipsoid(1, (2.0, 1.0, 0.5)), "jitter": meshes.perturbed(*meshes.icosphere(1), 0.1, 3)}


@pytest.mark.parametrize("name", list(MESHES))
def test_topology_bit_exact(lib, name):
    from oracle.topology import Topology
    from paper_2312_06367_gb300 import Solver
    V, F = MESHES[name]
    s = Solver(V, F, dt=0.3, nt=5)
    t = Topology(V, F)
    E, cp, cm = s.topology()
    assert np.array_equal(E, t.E) and np.array_equal(cp, t.cplus) and np.array_equal(cm, t.cminus)
    assert (s.ne, s.nc, s.nv, s.genus) == (t.ne, t.nc, t.nv, t.genus)
    assert s.D == t.D
    from oracle.topology import n_lags
    assert s.K == n_lags(t.D, 0.3)


@pytest.mark.parametrize("name", list(MESHES))
def test_bc_table_matches_oracle(lib, name):
    from oracle.bc import BarycentricBC
    from oracle.topology import Topology
    from paper_2312_06367_gb300 import Solver
    V, F = MESHES[name]
    s = Solver(V, F, dt=0.3, nt=5)
    b = BarycentricBC(Topology(V, F))
    ft, fn, ph, fV, fF = s.bc_table()
    assert np.array_equal(fF, b.fF)
    assert np.max(np.abs(fV - b.fV)) == 0.0
    ref_ft = np.repeat(np.arange(b.nf), np.diff(b.bc_ptr))
    assert np.array_equal(ft, ref_ft) and np.array_equal(fn, b.bc_fn)
    assert np.max(np.abs(ph - b.bc_phi)) < 1e-15


def test_rejects_bad_meshes(lib):
    from paper_2312_06367_gb300 import Solver, TdcfieError
    V, F = meshes.icosphere(1)
    with pytest.raises(TdcfieError, match="E_MESH"):
        Solver(V, F[:-1], dt=0.3, nt=5)                      # open surface
    Fb = F.copy()
    Fb[0] = Fb[0][[0, 2, 1]]
    with pytest.raises(TdcfieError, match="E_MESH"):
        Solver(V, Fb, dt=0.3, nt=5)                          # inconsistent orientation
    V2, F2 = meshes.icosphere(0)
    with pytest.raises(TdcfieError, match="E_MESH"):
        Solver(np.concatenate([V, V2]), np.concatenate([F, F2 + V.shape[0]]), dt=0.3, nt=5)   # disconnected
    with pytest.raises(TdcfieError, match="E_ARG"):
        Solver(V, F, dt=-1.0, nt=5)
    with pytest.raises(TdcfieError, match="E_UNSUPPORTED"):
        Solver(V, F, dt=0.3, nt=5, precision="fp32", R=16)


def test_time_order_sets_the_lag_count(lib):
    """K = ceil(D/dt + order + 1): q_0 is supported on [-dt, (order + 1) dt] (host only)."""
    from oracle.topology import Topology, n_lags
    from paper_2312_06367_gb300 import Solver, TdcfieError
    V, F = meshes.icosphere(1)
    D = Topology(V, F).D
    for order in (1, 2):
        s = Solver(V, F, dt=0.3, nt=5, time_order=order)
        assert s.K == n_lags(D, 0.3, order) == int(np.ceil(D / 0.3 + order + 1))
    with pytest.raises(TdcfieError, match="E_ARG"):
        Solver(V, F, dt=0.3, nt=5, time_order=3)
