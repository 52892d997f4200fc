"""GPU parity: the CUDA path through the C ABI against the FP64 oracle, same seeded inputs.

Tolerances (the accuracy bars of the two path classes): FP64 path rel-L2 <= 1e-10, reduced precision <= 1e-5
on the surface current j (all steps x edges x right-hand sides); assembled FP64 matrices per block
within 1e-10 relative Frobenius (atomic summation order only).
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
    y = mot.march_factored(fm, fm.rhs(e, h))
    return ops, fm, fm.postprocess(y)           # (nt, ne, R)


def _gpu(V, F, dt, nt, pw, precision="fp64", alpha=1.0):
    import torch
    from paper_2312_06367_gb300 import Solver
    R = pw["k"].shape[0]
    s = Solver(V, F, dt=dt, nt=nt, alpha=alpha, precision=precision, R=R).assemble()
    out = torch.zeros((nt, R, s.ne), dtype=s.dtype, device="cuda")
    s.march(pw, out)
    torch.cuda.synchronize()
    return s, out.double().cpu().numpy().transpose(0, 2, 1)   # (nt, ne, R)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def ico1():
    V, F = meshes.icosphere(1)
    pw = excitation.random_batch(3, seed=11, t0=4.0, sigma=1.5)
    ops, fm, j = _oracle(V, F, 0.4, 40, pw)
    return V, F, pw, ops, fm, j


def test_assembled_blocks_match_oracle(ico1):
    V, F, pw, ops, fm, _ = ico1
    from paper_2312_06367_gb300 import Solver
    s = Solver(V, F, dt=0.4, nt=40).assemble()
    checks = [("G", ops.G), ("Zs", ops.Zs), ("Zh", ops.Zh), ("M", ops.M), ("PS", fm.PS), ("L1", fm.L1),
              ("L2", fm.L2)]
    for k in range(ops.K):
        checks += [(("S", k), ops.S[k]), (("H", k), ops.H[k]), (("MM", k), ops.MM[k]), (("T", k), fm.T(k))]
    worst = 0.0
    for key, ref in checks:
        name, k = (key, 0) if isinstance(key, str) else key
        got = s.matrix(name, k)
        nref = np.linalg.norm(ref)
        if nref == 0.0:
            assert np.max(np.abs(got)) < 1e-14
            continue
        e = np.linalg.norm(got - ref) / nref
        worst = max(worst, e)
        assert e < 1e-10, (key, e)
    print("worst block rel err", worst)


def test_fp64_march_small_batch(ico1):
    V, F, pw, ops, fm, j_ref = ico1
    _, j = _gpu(V, F, 0.4, 40, pw, "fp64")
    assert rel(j, j_ref) < 1e-10


def test_fp32_march_small_batch(ico1):
    V, F, pw, ops, fm, j_ref = ico1
    _, j = _gpu(V, F, 0.4, 40, pw, "fp32")
    assert rel(j, j_ref) < 1e-5


def test_batch_equals_single(ico1):
    """R incident waves marched together give the same currents as one at a time (FP64)."""
    V, F, pw, *_ = ico1
    _, jb = _gpu(V, F, 0.4, 20, pw, "fp64")
    for r in range(3):
        one = {k: v[r:r + 1] for k, v in pw.items()}
        _, j1 = _gpu(V, F, 0.4, 20, one, "fp64")
        assert rel(jb[:, :, r:r + 1], j1) < 1e-13


def test_step_api_resume_matches_march(ico1):
    """Stepping in chunks continues the same march (state persists across calls)."""
    import torch
    from paper_2312_06367_gb300 import Solver
    V, F, pw, *_ = ico1
    s = Solver(V, F, dt=0.4, nt=30, R=3).assemble()
    full = torch.zeros((30, 3, s.ne), dtype=torch.float64, device="cuda")
    s.march(pw, full)
    s.set_excitation(pw)
    parts = torch.zeros_like(full)
    s.step(7, parts[:7])
    s.step(0, None)
    s.step(13, parts[7:20])
    s.step(10, parts[20:])
    torch.cuda.synchronize()
    assert torch.equal(full, parts)


def test_host_output_march(ico1):
    from paper_2312_06367_gb300 import Solver
    V, F, pw, ops, fm, j_ref = ico1
    s = Solver(V, F, dt=0.4, nt=40, R=3).assemble()
    out = np.zeros((40, 3, s.ne))
    s.march(pw, out, out_on_host=True)
    assert rel(out.transpose(0, 2, 1), j_ref) < 1e-10


def test_sphere480_fp64_full_workload():
    """The 480-edge sphere workload, 300 FP64 steps, end to end vs the oracle (<= 1e-10)."""
    w = workloads.sphere480_fp64()
    _, _, j_ref = _oracle(w["V"], w["F"], w["dt"], w["Nt"], w["pw"])
    _, j = _gpu(w["V"], w["F"], w["dt"], w["Nt"], w["pw"], "fp64")
    assert rel(j, j_ref) < 1e-10


def test_torus_fp32_small():
    V, F = meshes.torus(1.0, 0.4, 12, 6)
    pw = excitation.single(t0=4.0, sigma=1.5)
    _, _, j_ref = _oracle(V, F, 0.5, 60, pw)
    _, j = _gpu(V, F, 0.5, 60, pw, "fp32")
    assert rel(j, j_ref) < 1e-5


@pytest.mark.parametrize("dtype,tol", [("float64", 1e-13), ("float32", 1e-5)])
@pytest.mark.parametrize("nblk,n,R", [(1, 1, 1), (13, 480, 1), (5, 97, 3), (42, 300, 8)])
def test_block_gemv_matches_numpy(dtype, tol, nblk, n, R):
    """Stand-alone history-sum entry point against a plain numpy FP64 evaluation."""
    import torch
    from paper_2312_06367_gb300 import block_gemv
    rng = np.random.default_rng(nblk * 1000 + n + R)
    B = rng.standard_normal((nblk, n, n))
    X = rng.standard_normal((nblk, R, n))
    ref = np.einsum("qij,qrj->ri", B, X)
    td = getattr(torch, dtype)
    out = block_gemv(torch.tensor(B, dtype=td, device="cuda"), torch.tensor(X, dtype=td, device="cuda"))
    torch.cuda.synchronize()
    got = out.double().cpu().numpy()
    assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref)


def test_replan_changes_precision_and_batch(ico1):
    """One FP64 assembly, three plans: FP64 R=3, FP32 R=1 (the second wave alone), FP64 R=3 again."""
    import torch
    from paper_2312_06367_gb300 import Solver
    V, F, pw, ops, fm, j_ref = ico1
    s = Solver(V, F, dt=0.4, nt=40, R=3).assemble()
    out = torch.zeros((40, 3, s.ne), dtype=torch.float64, device="cuda")
    s.march(pw, out)
    torch.cuda.synchronize()
    assert rel(out.cpu().numpy().transpose(0, 2, 1), j_ref) < 1e-10
    s.replan("fp32", 1)
    one = {k: v[1:2] for k, v in pw.items()}
    o1 = torch.zeros((40, 1, s.ne), dtype=torch.float32, device="cuda")
    s.march(one, o1)
    torch.cuda.synchronize()
    assert rel(o1.double().cpu().numpy().transpose(0, 2, 1), j_ref[:, :, 1:2]) < 1e-5
    s.replan("fp64", 3)
    out2 = torch.zeros_like(out)
    s.march(pw, out2)
    torch.cuda.synchronize()
    assert torch.equal(out, out2)
