"""Factored history form (Sec. IV-A, Eq. dis_TD_CFIE; Sec. IV-B) through the C ABI against the
FP64 oracle's factored march (oracle/mot.py:march_factored), on the same seeded inputs.

* The compressed shells hold exactly the nonzeros of S_k, MM_k + G/2 [k = 0] and Phi_k (k >= 1) of
  the device's own FP64 assembly: integer count, bit-exact.
* FP64 factored path: rel-L2 <= 1e-10 on the current j (the 480-edge sphere at its configured
  dt 0.2 and 300 steps, and a 3-wave batch on the 120-edge sphere).
* FP32 factored path: <= 1e-5 (the 864-edge torus at dt 2.0 over 1000 steps; 5 waves on the
  120-edge sphere, the ragged R of the 8-wave kernels).
* Both forms on the GPU agree to FP64 rounding on a many-lag case (1920 edges, dt 0.05, K = 42), and
  the factored form streams fewer bytes per step there.
* Refusals: tensor-core precision, GMRES; a batch with a factored member steps it bit for bit.
"""
import numpy as np
import pytest

from synth import excitation, meshes, workloads

pytestmark = pytest.mark.gpu


def _oracle(V, F, dt, nt, pw, alpha=1.0):
    from oracle import mot, rhs
    from oracle.assemble import Operators
    from oracle.formulation import Formulation
    ops = Operators(V, F, dt=dt, alpha=alpha)
    fm = Formulation(ops)
    e, h = rhs.incident_tests(ops, pw, dt * np.arange(1, nt + 1))
    return fm.postprocess(mot.march_factored(fm, fm.rhs(e, h)))     # (nt, ne, R)


def _march(s, pw, nt):
    import torch
    R = pw["k"].shape[0]
    out = torch.zeros((nt, R, s.ne), dtype=s.dtype, device="cuda")
    s.march(pw, out)
    torch.cuda.synchronize()
    return out.double().cpu().numpy().transpose(0, 2, 1)


def _solver(V, F, dt, nt, pw, precision, alpha=1.0, form="factored"):
    from paper_2312_06367_gb300 import Solver
    s = Solver(V, F, dt=dt, nt=nt, alpha=alpha, precision=precision, R=pw["k"].shape[0]).assemble()
    if form != "dense":
        s.set_history_form(form)
    return s


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def ico1():
    V, F = meshes.icosphere(1)
    pw = excitation.random_batch(5, seed=17, t0=4.0, sigma=1.5)
    return V, F, pw, _oracle(V, F, 0.4, 40, pw)


def test_shell_nonzeros_bit_exact(ico1):
    V, F, pw, _ = ico1
    s = _solver(V, F, 0.4, 40, excitation.single(t0=4.0, sigma=1.5), "fp64")
    G = s.matrix("G")
    want = 0
    for k in range(s.K):
        want += np.count_nonzero(s.matrix("S", k))
        want += np.count_nonzero(s.matrix("MM", k) + (0.5 * G if k == 0 else 0.0))
        if k >= 1:
            want += np.count_nonzero(s.matrix("Phi", k))
    st = s.history_stats()
    print(f"120 edges, K = {s.K}: shell nonzeros {st['nnz']} of {(2 * s.K * s.ne ** 2 + (s.K - 1) * s.nc ** 2)}")
    assert st["form"] == "factored"
    assert st["nnz"] == want


def test_fp64_factored_three_waves(ico1):
    V, F, pw, j_ref = ico1
    pw3 = {k: v[:3] for k, v in pw.items()}
    s = _solver(V, F, 0.4, 40, pw3, "fp64")
    err = rel(_march(s, pw3, 40), j_ref[..., :3])
    print(f"FP64 factored, 120 edges, R = 3: rel-L2 vs oracle {err:.2e}")
    assert err < 1e-10


def test_fp32_factored_five_waves(ico1):
    V, F, pw, j_ref = ico1
    s = _solver(V, F, 0.4, 40, pw, "fp32")
    err = rel(_march(s, pw, 40), j_ref)
    print(f"FP32 factored, 120 edges, R = 5: rel-L2 vs oracle {err:.2e}")
    assert err < 1e-5


def test_fp64_factored_sphere480_full_workload():
    w = workloads.sphere480_fp64()
    j_ref = _oracle(w["V"], w["F"], w["dt"], w["Nt"], w["pw"])
    s = _solver(w["V"], w["F"], w["dt"], w["Nt"], w["pw"], "fp64")
    assert s.ne == 480
    err = rel(_march(s, w["pw"], w["Nt"]), j_ref)
    print(f"FP64 factored, sphere 480 edges, dt {w['dt']}, {w['Nt']} steps: rel-L2 vs oracle {err:.2e}")
    assert err < 1e-10


def test_fp32_factored_torus864_full_workload():
    w = workloads.torus864_fp32()
    alpha = 0.5          # as in the dense torus test: alpha = 1 has a growing mode at this dt
    j_ref = _oracle(w["V"], w["F"], w["dt"], w["Nt"], w["pw"], alpha)
    s = _solver(w["V"], w["F"], w["dt"], w["Nt"], w["pw"], "fp32", alpha=alpha)
    j = _march(s, w["pw"], w["Nt"])
    err = rel(j, j_ref)
    late = np.abs(j[-200:]).max() / np.abs(j).max()
    print(f"FP32 factored, torus 864 edges, dt 2.0, 1000 steps: rel-L2 vs oracle {err:.2e}, late/peak {late:.1e}")
    assert err < 1e-5
    assert late < 1e-6


def test_forms_agree_many_lags_and_bytes():
    V, F = meshes.icosphere(3)
    pw = excitation.random_batch(2, seed=5, t0=3.0, sigma=1.0)
    nt = 200
    d = _solver(V, F, 0.05, nt, pw, "fp64", form="dense")
    assert d.ne == 1920 and d.K >= 40
    jd = _march(d, pw, nt)
    sd = d.history_stats()
    d.set_history_form("factored")
    jf = _march(d, pw, nt)
    sf = d.history_stats()
    err = rel(jf, jd)
    print(f"1920 edges, K = {d.K}: factored vs dense rel-L2 {err:.2e}; matrix bytes per step "
          f"dense {sd['step_bytes'] / 1e6:.0f} MB, factored {sf['step_bytes'] / 1e6:.0f} MB "
          f"(shell nonzeros {sf['nnz'] / d.ne ** 2:.2f} ne^2)")
    assert err < 1e-11
    assert sf["step_bytes"] < 0.7 * sd["step_bytes"]
    # and back to the dense form on the same handle
    d.set_history_form("dense")
    assert d.history_stats()["form"] == "dense"
    assert np.array_equal(_march(d, pw, nt), jd)


def test_refusals():
    from paper_2312_06367_gb300 import Solver, TdcfieError
    V, F = meshes.icosphere(1)
    s = Solver(V, F, dt=0.4, nt=10, precision="fp32").assemble()
    s.set_solver("gmres", "prev", 1e-8)
    with pytest.raises(TdcfieError, match="direct solve"):
        s.set_history_form("factored")
    s.set_solver("direct", "prev", 1e-8)
    s.set_history_form("factored")
    with pytest.raises(TdcfieError, match="direct solve"):
        s.set_solver("gmres", "prev", 1e-8)
    V2, F2 = meshes.icosphere(2)
    t = Solver(V2, F2, dt=0.2, nt=10, precision="fp16x3", R=64).assemble()
    with pytest.raises(TdcfieError, match="FP64 and FP32"):
        t.set_history_form("factored")


def test_batch_with_factored_member_is_bit_exact():
    import torch
    from paper_2312_06367_gb300 import Batch
    V, F = meshes.icosphere(1)
    V2, F2 = meshes.torus(1.0, 0.4, 12, 6)
    pw = excitation.single(t0=4.0, sigma=1.5)
    nt = 30
    a = _solver(V, F, 0.4, nt, pw, "fp64")
    b = _solver(V2, F2, 0.5, nt, pw, "fp32", form="dense")
    ja, jb = _march(a, pw, nt), _march(b, pw, nt)
    for s in (a, b):
        s.set_excitation(pw)
    outs = [torch.zeros((nt, 1, s.ne), dtype=s.dtype, device="cuda") for s in (a, b)]
    bt = Batch([a, b])
    assert bt.tune(1)["persistent"] == 0          # a factored member takes the graph-branch form
    bt.step(nt, outs)
    bt.close()
    torch.cuda.synchronize()
    for o, ref in zip(outs, (ja, jb)):
        assert np.array_equal(o.double().cpu().numpy().transpose(0, 2, 1), ref)
