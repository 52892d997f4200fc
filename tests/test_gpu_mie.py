"""GPU FP64 path against the Mie-series transient on two meshes: a convergence check.

The same pulse and time step as the oracle's Mie pin (dt 0.2, 300 steps); the 320- and
1280-triangle spheres are marched on the GPU (whose FP64 path matches the oracle to 1e-10 wherever
the oracle can assemble), and the error against the series must shrink under refinement."""
import numpy as np
import pytest

from mie_series import current_at, mie_current, points
from synth import excitation, meshes

pytestmark = pytest.mark.gpu


def _gpu_currents(level):
    import torch
    from oracle.topology import Topology
    from paper_2312_06367_gb300 import Solver
    V, F = meshes.icosphere(level)
    s = Solver(V, F, dt=0.2, nt=300).assemble()
    out = torch.zeros((300, 1, s.ne), dtype=torch.float64, device="cuda")
    s.march(excitation.single(t0=8.0, sigma=2.0), out)
    torch.cuda.synchronize()
    s.close()
    return Topology(V, F), out[:, 0, :].cpu().numpy()


def test_mie_error_shrinks_under_refinement():
    p = points()
    t = 0.2 * np.arange(1, 301)
    J_mie = mie_current(p, t)
    errs = []
    for level in (2, 3):
        topo, j = _gpu_currents(level)
        J = current_at(topo, j, p)
        errs.append(np.linalg.norm(J - J_mie) / np.linalg.norm(J_mie))
    print(f"MOT (GPU FP64) vs Mie: 320 triangles {errs[0]:.3f}, 1280 triangles {errs[1]:.3f}")
    assert errs[0] < 0.15 and errs[1] < errs[0]
