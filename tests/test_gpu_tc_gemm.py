"""The split-precision tensor-core product by itself (tdcfie_tc_gemm), against plain FP64 numpy.

out[r][i] = sum_q sum_j A_q[i][j] x_q[r][j] is the history sum of the MOT recurrence (Sec. IV-B,
the sum over k of T_k y_{n-k}).  Two references:
  * the FP64 product of the given operands: the error is then the storage of the split operands,
    bounded entry by entry by the split's precision times sum_j |A_ij| |x_j|;
  * the FP64 product of the split operands themselves (the same power-of-two scales and 16-bit
    roundings, written out in numpy): what is left is the tensor-core accumulation, a few FP32
    roundings of each 64-wide k tile's partial sum.
Sizes cover one element, ragged row and column tiles, CTAs whose stream-K range spans two row
tiles, a history-like stack and a full 7680-edge block.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

FP16X3, BF16X3 = 3, 2


def _pow2_scale(m):
    """power of two p with m p in [2^13, 2^14), exponent clamped to +-100, 1 for m == 0."""
    m = np.asarray(m, dtype=np.float32)
    out = np.ones(m.shape, dtype=np.float64)
    pos = (m > 0) & np.isfinite(m)
    _, e = np.frexp(m[pos])
    out[pos] = np.ldexp(1.0, np.clip(14 - e, -100, 100))
    return out


def _round16(v, fp16):
    import torch
    f = np.asarray(v, dtype=np.float64).astype(np.float32)
    if fp16:
        return f.astype(np.float16).astype(np.float64)
    return torch.from_numpy(f).to(torch.bfloat16).to(torch.float64).numpy()


def _slices(v, n, fp16):
    out = []
    for _ in range(n):
        s = _round16(v, fp16)
        out.append(s)
        v = v - s
    return out


def split_reference(A, X, fp16):
    """The product of the stored split operands (products the kernel forms), in FP64."""
    nblk, rows, cols = A.shape
    ld = (cols + 63) // 64 * 64
    # one power-of-two scale per row, common to all blocks
    sa = _pow2_scale(np.max(np.abs(A), axis=(0, 2)).astype(np.float32))[None, :].repeat(nblk, 0)   # (q, rows)
    ah, al = _slices(A * sa[:, :, None], 2, fp16)
    Xp = np.zeros((nblk, X.shape[1], ld))
    Xp[:, :, :cols] = X
    t = Xp.reshape(nblk, X.shape[1], ld // 64, 64)
    sx = _pow2_scale(np.max(np.abs(t.astype(np.float32)), axis=3))           # (q, R, tiles)
    xs = _slices(t * sx[..., None], 3 if fp16 else 2, fp16)
    xs = [(s / sx[..., None]).reshape(nblk, X.shape[1], ld)[:, :, :cols] for s in xs]
    ah, al = ah / sa[:, :, None], al / sa[:, :, None]
    pairs = [(ah, xs[0]), (ah, xs[1]), (al, xs[0])]
    if fp16:
        pairs += [(ah, xs[2]), (al, xs[1])]
    return sum(np.einsum("qij,qrj->ri", a, x) for a, x in pairs)


def _run(A, X, prec):
    import torch
    from paper_2312_06367_gb300 import tc_gemm
    out = tc_gemm(torch.tensor(A, device="cuda"), torch.tensor(X, device="cuda"), prec)
    torch.cuda.synchronize()
    return out.cpu().numpy()


CASES = [(1, 1, 1), (3, 300, 200), (2, 130, 70), (5, 1000, 512), (43, 480, 480)]


@pytest.mark.parametrize("prec,bits", [(FP16X3, 21), (BF16X3, 14)])
@pytest.mark.parametrize("nblk,rows,cols", CASES)
def test_tc_gemm_matches_fp64(prec, bits, nblk, rows, cols):
    rng = np.random.default_rng(nblk * 7919 + rows * 31 + cols)
    A = rng.standard_normal((nblk, rows, cols))
    X = rng.standard_normal((nblk, 64, cols))
    ref = np.einsum("qij,qrj->ri", A, X)
    mag = np.einsum("qij,qrj->ri", np.abs(A), np.abs(X))
    got = _run(A, X, prec)
    err = np.abs(got - ref)
    print(f"prec {prec} {nblk}x{rows}x{cols}: max err / (|A||x|) = {np.max(err / mag):.2e}, "
          f"rel-L2 {np.linalg.norm(got - ref) / np.linalg.norm(ref):.2e}")
    assert np.all(err <= 2.0 ** -bits * mag + 1e-300)


@pytest.mark.parametrize("prec", [FP16X3, BF16X3])
@pytest.mark.parametrize("nblk,rows,cols", CASES[1:])
def test_tc_gemm_accumulation(prec, nblk, rows, cols):
    """Against the product of the split operands: only the tensor-core accumulation is left."""
    rng = np.random.default_rng(nblk * 104729 + rows + cols)
    A = rng.standard_normal((nblk, rows, cols))
    X = rng.standard_normal((nblk, 64, cols))
    ref = split_reference(A, X, prec == FP16X3)
    got = _run(A, X, prec)
    mag = np.einsum("qij,qrj->ri", np.abs(A), np.abs(X))
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    worst = np.max(np.abs(got - ref) / mag)
    print(f"prec {prec} {nblk}x{rows}x{cols}: accumulation rel-L2 {rel:.2e}, max / (|A||x|) {worst:.2e}")
    # FP32 accumulation of each k tile's products is about 2^-24 of the tile's partial; a dropped
    # product or a wrong scale would show as 2^-11 or worse
    assert rel < 4 * 2.0 ** -24
    assert worst < 2.0 ** -21


def test_tc_gemm_wide_range_and_zero_tiles():
    """Rows spanning 20 orders of magnitude (one row scale serves both blocks), an all-zero vector
    tile and a tiny (1e-30) tile."""
    rng = np.random.default_rng(5)
    nblk, rows, cols = 2, 256, 320
    A = rng.standard_normal((nblk, rows, cols)) * 10.0 ** rng.uniform(-10, 10, (nblk, rows, cols))
    X = rng.standard_normal((nblk, 64, cols))
    X[0, :, 64:128] = 0.0
    X[1, :, 128:192] *= 1e-30
    ref = np.einsum("qij,qrj->ri", A, X)
    mag = np.einsum("qij,qrj->ri", np.abs(A), np.abs(X))
    got = _run(A, X, FP16X3)
    assert np.all(np.abs(got - ref) <= 2.0 ** -21 * mag)


def test_tc_gemm_full_block_deterministic():
    """One 7680 x 7680 block (the 7680-edge solve's size): FP64 agreement and bit-identical repeats."""
    rng = np.random.default_rng(7680)
    A = rng.standard_normal((1, 7680, 7680)) / 7680 ** 0.5
    X = rng.standard_normal((1, 64, 7680))
    ref = np.einsum("qij,qrj->ri", A, X)
    mag = np.einsum("qij,qrj->ri", np.abs(A), np.abs(X))
    g1 = _run(A, X, FP16X3)
    g2 = _run(A, X, FP16X3)
    assert np.array_equal(g1, g2)
    assert np.all(np.abs(g1 - ref) <= 2.0 ** -21 * mag)
    print(f"7680 block: rel-L2 vs FP64 {np.linalg.norm(g1 - ref) / np.linalg.norm(ref):.2e}")


def test_tc_gemm_rejects_bad_arguments():
    import torch
    from paper_2312_06367_gb300 import TdcfieError, tc_gemm
    A = torch.zeros((1, 8, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(TdcfieError):
        tc_gemm(A, torch.zeros((1, 32, 8), dtype=torch.float64, device="cuda"))      # R != 64
    with pytest.raises(TdcfieError):
        tc_gemm(A, torch.zeros((1, 64, 8), dtype=torch.float64, device="cuda"), precision=1)   # FP32
