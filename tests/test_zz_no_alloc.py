"""The history-sum entry point that allocates nothing (tdcfie_block_gemv_noalloc).

It serves callers that cannot allocate device memory at call time (another thread holding a
global-mode stream capture, an allocator that has reserved the device memory, a loop that cannot
take an allocation's synchronisation).  Its partial sums live in a static device array shared by
all calls.  Two calls in a row with different inputs must each match the allocating entry point
(tdcfie_block_gemv) within the tolerances of the history-sum tests; sizes beyond the static
array are refused with an error.  This file sorts last so that a run stopping at the first
failure has run every other test first; it also passes alone in a fresh process."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _inputs(seed, nblk, n, R, dtype):
    import torch
    rng = np.random.default_rng(seed)
    td = getattr(torch, dtype)
    B = torch.tensor(rng.standard_normal((nblk, n, n)), dtype=td, device="cuda")
    X = torch.tensor(rng.standard_normal((nblk, R, n)), dtype=td, device="cuda")
    return B, X


@pytest.mark.parametrize("dtype,tol", [("float64", 1e-13), ("float32", 1e-5)])
def test_noalloc_matches_allocating_entry_point_on_two_calls(dtype, tol):
    import torch
    from paper_2312_06367_gb300 import block_gemv, block_gemv_noalloc
    for seed, (nblk, n, R) in ((1, (42, 300, 8)), (2, (13, 480, 1))):
        B, X = _inputs(seed, nblk, n, R, dtype)
        ref = block_gemv(B, X)
        out = torch.full((R, n), float("nan"), dtype=B.dtype, device="cuda")
        block_gemv_noalloc(B, X, out)
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        err = torch.linalg.norm(out.double() - ref.double()) / torch.linalg.norm(ref.double())
        assert float(err) <= tol


def test_noalloc_rejects_sizes_beyond_its_static_scratch():
    import torch
    from paper_2312_06367_gb300 import TdcfieError, block_gemv_noalloc
    # 64 x 8 x 8193 FP64 partial sums = 4194816 > 4194304
    B = torch.zeros((64, 8193, 1), dtype=torch.float64, device="cuda").expand(64, 8193, 8193)
    X = torch.zeros((64, 8, 8193), dtype=torch.float64, device="cuda")
    out = torch.zeros((8, 8193), dtype=torch.float64, device="cuda")
    with pytest.raises(TdcfieError, match="E_ARG"):
        block_gemv_noalloc(B, X, out)
