"""Reduced-precision paths at a small time step (dt = 0.05, 42 blocks), where the MOT
post-processing (y_n - y_{n-1}) / dtt (Eq. post_processing) magnifies any per-step error of y by
about |y| / |y_n - y_{n-1}| (about 20 here).

The FP32 path accumulates every row dot product error-free (FMA product errors and TwoSum), so its
remaining error is the FP32 storage of blocks and vectors: it must meet the reduced-precision bar,
rel-L2 <= 1e-5, against the FP64 oracle (480 edges) and against the oracle-verified FP64 GPU path
(1920 edges, where the oracle assembly takes too long for a test).  The tensor-core FP16X3 path
accumulates in the tensor cores' FP32 accumulator; its error here is measured and bounded by the
value recorded with the design notes (it does not meet 1e-5 at this time step)."""
import numpy as np
import pytest

from synth import excitation, meshes

pytestmark = pytest.mark.gpu

DT = 0.05
PW = excitation.fibonacci_batch(64, seed=2312063670, t0=8.0, sigma=1.0)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _gpu(level, nt, precision, R):
    import torch
    from paper_2312_06367_gb300 import Solver
    V, F = meshes.icosphere(level)
    pw = {k: v[:R] for k, v in PW.items()}
    s = Solver(V, F, dt=DT, nt=nt, precision=precision, R=R).assemble()
    out = torch.zeros((nt, R, s.ne), dtype=s.dtype, device="cuda")
    s.march(pw, out)
    torch.cuda.synchronize()
    s.close()
    return out.double().cpu().numpy().transpose(0, 2, 1)      # (nt, ne, R)


@pytest.fixture(scope="module")
def ico2_oracle():
    from oracle import mot, rhs
    from oracle.assemble import Operators
    from oracle.formulation import Formulation
    V, F = meshes.icosphere(2)
    pw = {k: v[:4] for k, v in PW.items()}
    ops = Operators(V, F, dt=DT)
    fm = Formulation(ops)
    e, h = rhs.incident_tests(ops, pw, DT * np.arange(1, 401))
    return fm.postprocess(mot.march_factored(fm, fm.rhs(e, h)))


def test_fp32_small_dt_480_edges_vs_oracle(ico2_oracle):
    err = rel(_gpu(2, 400, "fp32", 4), ico2_oracle)
    print(f"fp32, 480 edges, dt 0.05: rel-L2 {err:.2e}")
    assert err < 1e-5


def test_fp32_small_dt_1920_edges_vs_fp64_path():
    ref = _gpu(3, 300, "fp64", 4)
    err = rel(_gpu(3, 300, "fp32", 4), ref)
    print(f"fp32, 1920 edges, dt 0.05: rel-L2 {err:.2e}")
    assert err < 1e-5


def test_fp16x3_small_dt_480_edges_measured(ico2_oracle):
    j = _gpu(2, 400, "fp16x3", 64)[:, :, :4]
    err = rel(j, ico2_oracle)
    print(f"fp16x3, 480 edges, dt 0.05: rel-L2 {err:.2e}")
    assert np.all(np.isfinite(j)) and err < 1e-4
