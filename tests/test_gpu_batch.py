"""GPU: several uneven scatterers stepped by one graph launch per step (tdcfie_batch_*).

Each member computes exactly what tdcfie_step computes on its own handle, so the batched currents
must equal the individually marched ones bit for bit, for mixed sizes, time steps, path precisions
and wave counts; one member is also held to the FP64 oracle."""
import numpy as np
import pytest

from synth import excitation, meshes

pytestmark = pytest.mark.gpu

CASES = [  # mesh, dt, precision, waves
    (meshes.icosphere(1), 0.4, "fp64", 3),
    (meshes.torus(1.0, 0.4, 12, 6), 0.5, "fp32", 1),
    (meshes.ellipsoid(2, (1.5, 1.0, 0.7)), 0.3, "fp64", 2),
    (meshes.icosphere(2), 0.2, "fp32", 4),
]
NT = 30


def _pw(i, R):
    return excitation.random_batch(R, seed=500 + i, t0=4.0, sigma=1.5)


def _solvers():
    from paper_2312_06367_gb300 import Solver
    out = []
    for i, ((V, F), dt, prec, R) in enumerate(CASES):
        s = Solver(V, F, dt=dt, nt=NT, precision=prec, R=R).assemble()
        s.set_excitation(_pw(i, R))
        out.append(s)
    return out


def test_batch_equals_individual_marches():
    import torch
    from paper_2312_06367_gb300 import Batch
    ss = _solvers()
    outs = [torch.zeros((NT, s.R, s.ne), dtype=s.dtype, device="cuda") for s in ss]
    b = Batch(ss)
    b.step(10, [o[:10] for o in outs])
    b.step(NT - 10, [o[10:] for o in outs])
    t = b.timing()
    b.close()
    torch.cuda.synchronize()
    for i, s in enumerate(ss):
        ref = torch.zeros_like(outs[i])
        s.march(_pw(i, s.R), ref)
        torch.cuda.synchronize()
        assert torch.equal(outs[i], ref), i
    assert t["step_ms"] > 0 and t["launches"] > 0


def test_batch_member_matches_oracle():
    import torch
    from oracle import mot, rhs
    from oracle.assemble import Operators
    from oracle.formulation import Formulation
    from paper_2312_06367_gb300 import Batch
    ss = _solvers()
    outs = [torch.zeros((NT, s.R, s.ne), dtype=s.dtype, device="cuda") for s in ss]
    b = Batch(ss)
    b.step(NT, outs)
    b.close()
    torch.cuda.synchronize()
    (V, F), dt, _, R = CASES[0]
    ops = Operators(V, F, dt=dt)
    fm = Formulation(ops)
    e, h = rhs.incident_tests(ops, _pw(0, R), dt * np.arange(1, NT + 1))
    j_ref = fm.postprocess(mot.march_factored(fm, fm.rhs(e, h)))
    j = outs[0].cpu().numpy().transpose(0, 2, 1)
    assert np.linalg.norm(j - j_ref) / np.linalg.norm(j_ref) < 1e-10


def test_batch_rejects_bad_input():
    from paper_2312_06367_gb300 import Batch, Solver, TdcfieError
    V, F = meshes.icosphere(1)
    s = Solver(V, F, dt=0.4, nt=5)
    with pytest.raises(TdcfieError):
        Batch([s])                       # not assembled
    s.assemble()
    with pytest.raises(TdcfieError):
        Batch([s, s])                    # twice
    b = Batch([s])
    with pytest.raises(TdcfieError):
        b.step(1)                        # no excitation
    b.close()


# ---------------------------------------------------------------- persistent form
# every member FP32 with one wave and the direct solve: one cooperative kernel per step
PCASES = [  # mesh, dt (uneven sizes and lags; a torus; one mesh whose edge count is not a multiple of 4)
    (meshes.icosphere(2), 0.2),
    (meshes.torus(1.0, 0.3, 16, 8), 0.3),
    (meshes.icosphere(1), 0.4),
    (meshes.ellipsoid(3, (1.8, 0.9, 0.6)), 0.25),
    (meshes.torus(1.0, 0.4, 10, 5), 0.5),
    (meshes.icosphere(3), 0.2),
]


def _psolvers(nt):
    from paper_2312_06367_gb300 import Solver
    out = []
    for i, ((V, F), dt) in enumerate(PCASES):
        s = Solver(V, F, dt=dt, nt=nt, precision="fp32", R=1).assemble()
        s.set_excitation(_pw(100 + i, 1))
        out.append(s)
    return out


def test_persistent_batch_equals_individual_marches():
    import torch
    from paper_2312_06367_gb300 import Batch
    nt = 40
    ss = _psolvers(nt)
    assert any(s.ne % 4 for s in ss) and len({s.K for s in ss}) > 2
    seq = 0.0                                         # the members stepped one after another
    for s in ss:
        s.step(3)
        s.step(10)
        seq += s.timing()["step_ms"]
        s.set_excitation(_pw(100 + ss.index(s), 1))
    b = Batch(ss)
    cfg = b.tune(2)
    assert cfg["persistent"] == 1
    outs = [torch.zeros((nt, 1, s.ne), dtype=torch.float32, device="cuda") for s in ss]
    b.step(15, [o[:15] for o in outs])
    b.step(nt - 15, [o[15:] for o in outs])
    t = b.timing()
    b.close()
    torch.cuda.synchronize()
    assert t["launches"] == 1
    for i, s in enumerate(ss):
        ref = torch.zeros_like(outs[i])
        s.march(_pw(100 + i, 1), ref)
        torch.cuda.synchronize()
        assert torch.isfinite(ref).all()
        assert torch.equal(outs[i], ref), i
    print(f"persistent batch of {len(ss)}: {t['step_ms']:.3f} ms per step (members one after another "
          f"{seq:.3f} ms), tuned {cfg}")


def test_persistent_batch_member_matches_oracle():
    import torch
    from oracle import mot, rhs
    from oracle.assemble import Operators
    from oracle.formulation import Formulation
    from paper_2312_06367_gb300 import Batch
    nt = 40
    ss = _psolvers(nt)
    outs = [torch.zeros((nt, 1, s.ne), dtype=torch.float32, device="cuda") for s in ss]
    b = Batch(ss)
    b.step(nt, outs)
    b.close()
    torch.cuda.synchronize()
    (V, F), dt = PCASES[1]
    ops = Operators(V, F, dt=dt)
    fm = Formulation(ops)
    e, h = rhs.incident_tests(ops, _pw(101, 1), dt * np.arange(1, nt + 1))
    j_ref = fm.postprocess(mot.march_factored(fm, fm.rhs(e, h)))
    j = outs[1].double().cpu().numpy().transpose(0, 2, 1)
    assert np.linalg.norm(j - j_ref) / np.linalg.norm(j_ref) < 1e-5
