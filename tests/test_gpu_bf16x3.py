"""Tensor-core (tcgen05) split-precision paths with 64 incident waves against the FP64 oracle.

Ragged sizes on purpose: 120 and 480 edges are not multiples of the 128-row tile, 80 and 320
triangles not multiples of 64.  FP16X3 must meet the reduced-precision bar, rel-L2 <= 1e-5 over
all steps x edges x waves.  BF16X3 stores about 2^-16 per entry and is held to 3e-4 (it measures
4.5e-5 on the 80-triangle sphere, as an FP64 emulation of the same splits predicts, and 1.1e-4 on
the 320-triangle sphere).  The runs go well past the pulse, so late steps see incident-field tests
that underflow FP32 (the fp16 scaling must stay finite there)."""
import numpy as np
import pytest

from synth import excitation, meshes

pytestmark = pytest.mark.gpu


def _oracle(V, F, dt, nt, pw):
    from oracle import mot, rhs
    from oracle.assemble import Operators
    from oracle.formulation import Formulation
    ops = Operators(V, F, dt=dt)
    fm = Formulation(ops)
    e, h = rhs.incident_tests(ops, pw, dt * np.arange(1, nt + 1))
    return fm.postprocess(mot.march_factored(fm, fm.rhs(e, h)))


def _tc(V, F, dt, nt, pw, precision):
    import torch
    from paper_2312_06367_gb300 import Solver
    s = Solver(V, F, dt=dt, nt=nt, precision=precision, R=64).assemble()
    out = torch.zeros((nt, 64, s.ne), dtype=torch.float32, device="cuda")
    s.march(pw, out)
    torch.cuda.synchronize()
    return out.double().cpu().numpy().transpose(0, 2, 1)


_CACHE = {}


@pytest.mark.parametrize("precision,bound", [("fp16x3", 1e-5), ("bf16x3", 3e-4)])
@pytest.mark.parametrize("level,dt,nt", [(1, 0.4, 40), (2, 0.2, 120)])
def test_tensor_core_path_matches_oracle(level, dt, nt, precision, bound):
    V, F = meshes.icosphere(level)
    pw = excitation.fibonacci_batch(64, seed=2312063670, t0=4.0, sigma=1.0)
    key = (level, dt, nt)
    if key not in _CACHE:
        _CACHE[key] = _oracle(V, F, dt, nt, pw)
    j_ref = _CACHE[key]
    j = _tc(V, F, dt, nt, pw, precision)
    err = np.linalg.norm(j - j_ref) / np.linalg.norm(j_ref)
    print(f"{precision} level {level}: rel-L2 {err:.3e}")
    assert np.all(np.isfinite(j))
    assert err < bound
