"""Failure detection, with every failure made on the host (no device fault, trap or hang).

* A GMRES per-step solve capped at one inner iteration cannot reach a 1e-12 residual: the step
  returns TDCFIE_E_NOCONV and names the first step that stopped above the tolerance.
* An unstable configuration (a polynomial eigenvalue outside the unit circle) grows until FP64
  overflows: the march stops with TDCFIE_E_NONFINITE at the step the mode's growth predicts.
* A NaN amplitude is refused by the host check before anything reaches the device.
"""
import re

import numpy as np
import pytest

from synth import excitation, meshes

pytestmark = pytest.mark.gpu


def _solver(**kw):
    from paper_2312_06367_gb300 import Solver
    V, F = meshes.icosphere(1)
    return Solver(V, F, dt=0.4, nt=40, **kw).assemble()


def test_gmres_cap_returns_noconv_with_step():
    import torch
    from paper_2312_06367_gb300 import TdcfieError
    s = _solver(solver="gmres", guess="zero", gmres_tol=1e-12, gmres_maxit=1, gmres_restart=1)
    pw = excitation.single(t0=4.0, sigma=1.5)
    s.set_excitation(pw)
    out = torch.zeros((5, 1, s.ne), dtype=torch.float64, device="cuda")
    with pytest.raises(TdcfieError, match="E_NOCONV") as ei:
        s.step(5, out)
    step = int(re.search(r"at step (\d+)", str(ei.value)).group(1))
    assert step == 1
    assert s.gmres_stats()["not_converged"] >= 1


def test_gmres_default_cap_converges():
    import torch
    s = _solver(solver="gmres", guess="prev", gmres_tol=1e-12)
    s.set_excitation(excitation.single(t0=4.0, sigma=1.5))
    out = torch.zeros((40, 1, s.ne), dtype=torch.float64, device="cuda")
    s.step(40, out)
    assert s.gmres_stats()["not_converged"] == 0


def test_unstable_mode_reports_its_overflow_step():
    """The 24 x 12 torus at dt 2.0 with alpha = 1 has a real polynomial eigenvalue near -1.89
    (outside the unit circle; the torus workload therefore runs at alpha 0.5).  Its mode grows
    until FP64 overflows; the march must stop with TDCFIE_E_NONFINITE at the step that the mode's
    growth, fitted on the finite steps, predicts."""
    import torch
    from paper_2312_06367_gb300 import Solver, TdcfieError
    V, F = meshes.torus(1.0, 0.4, 24, 12)
    nt = 1400
    s = Solver(V, F, dt=2.0, nt=nt, alpha=1.0, precision="fp64").assemble()
    out = torch.zeros((nt, 1, s.ne), dtype=torch.float64, device="cuda")
    with pytest.raises(TdcfieError, match="E_NONFINITE") as ei:
        s.march(excitation.single(t0=8.0, sigma=2.0), out)
    step = int(re.search(r"at step (\d+)", str(ei.value)).group(1))
    j = out[:, 0, :].abs().amax(dim=1).cpu().numpy()
    n = np.arange(1, nt + 1)
    sel = (n >= 300) & (n <= 700)
    slope, icpt = np.polyfit(n[sel], np.log(j[sel]), 1)
    n_pred = (np.log(np.finfo(np.float64).max) - icpt) / slope
    print(f"growth per step {np.exp(slope):.4f}; overflow predicted at {n_pred:.1f}, reported at step {step}")
    assert 1.8 < np.exp(slope) < 2.0
    assert np.all(np.isfinite(j[:step - 1]))
    assert abs(step - n_pred) <= 8


def test_nan_amplitude_is_refused_on_the_host():
    from paper_2312_06367_gb300 import TdcfieError
    s = _solver()
    pw = dict(excitation.single(t0=4.0, sigma=1.5), amp=np.array([np.nan]))
    with pytest.raises(TdcfieError, match="E_ARG"):
        s.set_excitation(pw)
