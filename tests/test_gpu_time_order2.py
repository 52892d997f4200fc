"""The higher-order temporal pair (shifted quadratic Lagrange h_i with q_i' = (h_i - h_{i+1})/dt,
the remark closing Sec. IV-B) on the GPU: opts.time_order = 2 against the oracle's order-2
assembly and march (oracle/quad.c, time order 2).

* Assembled retarded blocks S_k, MM_k, Phi_k: rel <= 1e-10 per block.
* FP64 march: rel-L2 <= 1e-10; FP32: <= 1e-5 (80-triangle sphere, 2 waves, dt 0.4, K = 8).
"""
import numpy as np
import pytest

from synth import excitation, meshes

pytestmark = pytest.mark.gpu

DT, NT = 0.4, 40


@pytest.fixture(scope="module")
def oracle_order2():
    from oracle import mot, rhs
    from oracle.assemble import Operators
    from oracle.formulation import Formulation
    V, F = meshes.icosphere(1)
    pw = excitation.random_batch(2, seed=23, t0=4.0, sigma=1.5)
    ops = Operators(V, F, dt=DT, time_order=2)
    fm = Formulation(ops)
    e, h = rhs.incident_tests(ops, pw, DT * np.arange(1, NT + 1))
    return V, F, pw, ops, fm.postprocess(mot.march_factored(fm, fm.rhs(e, h)))


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_order2_blocks_and_march_vs_oracle(oracle_order2):
    import torch
    from paper_2312_06367_gb300 import Solver
    V, F, pw, ops, j_ref = oracle_order2
    s = Solver(V, F, dt=DT, nt=NT, precision="fp64", R=2, time_order=2).assemble()
    assert s.K == ops.K == 8
    worst = 0.0
    for k in range(s.K):
        for name, ref in (("S", ops.S[k]), ("MM", ops.MM[k]), ("Phi", ops.Phi[k])):
            nref = np.linalg.norm(ref)
            if nref == 0.0:
                assert np.abs(s.matrix(name, k)).max() < 1e-14
                continue
            worst = max(worst, np.linalg.norm(s.matrix(name, k) - ref) / nref)
    out = torch.zeros((NT, 2, s.ne), dtype=torch.float64, device="cuda")
    s.march(pw, out)
    torch.cuda.synchronize()
    e64 = rel(out.cpu().numpy().transpose(0, 2, 1), j_ref)
    s.replan("fp32", 2)
    o32 = torch.zeros((NT, 2, s.ne), dtype=torch.float32, device="cuda")
    s.march(pw, o32)
    torch.cuda.synchronize()
    e32 = rel(o32.double().cpu().numpy().transpose(0, 2, 1), j_ref)
    print(f"time order 2: worst block rel err {worst:.1e}; march FP64 {e64:.2e}, FP32 {e32:.2e}")
    assert worst < 1e-10
    assert e64 < 1e-10
    assert e32 < 1e-5
