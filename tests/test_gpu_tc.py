"""The mixed form's tensor-core product (tcgen05, 3xTF32, FP32 accumulation)
against the FP64 product, element by element.

Shapes: the subspace-search products of the bench workload's zip-up cuts
(T is 256 x 4096, the search keeps 80 directions: 256 x 4096 x 80 and
80 x 256 x 4096), their transposed operand layouts, and ragged sizes that
span several 128-row tiles, several N tiles and a K tail that is not a
multiple of the 32-element K block.  The bound per element is the 3xTF32
split error (the dropped lo*lo term and the rounding of lo, 3 x 2^-22 of
|a||b| per product) plus FP32 accumulation over K terms, taken as
(K + 3) 2^-23 (|op(A)| |op(B)|)_ij.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2406_17823_b300 as P
    return P.Context(6)


CASES = [
    # M, N, K, transA, transB
    (256, 80, 4096, False, False),   # Y = T Z
    (80, 4096, 256, False, False),   # Z^T = Q^T T
    (256, 80, 4096, False, True),
    (80, 4096, 256, True, False),
    (300, 37, 1000, True, True),     # ragged in every dimension
    (129, 257, 33, False, False),
    (1, 1, 1, False, False),
    (4096, 4096, 4096, False, False),  # many full tiles (throughput shape)
]


@pytest.mark.parametrize("M,N,K,tA,tB", CASES)
def test_tc_gemm_within_3xtf32_bound(ctx, M, N, K, tA, tB):
    import torch
    rng = np.random.default_rng(M * 7919 + N * 31 + K)
    A = rng.standard_normal((K, M) if tA else (M, K))
    B = rng.standard_normal((N, K) if tB else (K, N))
    # rows of very different scale, as in a factor with a decaying spectrum
    if tA:
        A *= np.logspace(0, -6, M)[None, :]
    else:
        A *= np.logspace(0, -6, M)[:, None]
    opA = A.T if tA else A
    opB = B.T if tB else B
    want = opA @ opB
    bound = (K + 3) * 2.0 ** -23 * (np.abs(opA) @ np.abs(opB)) + 1e-300
    dA = torch.tensor(A, device="cuda")
    dB = torch.tensor(B, device="cuda")
    got = ctx.gemm_tf32x3(dA, dB, transA=tA, transB=tB).cpu().numpy()
    ratio = np.abs(got - want) / bound
    print(f"{M}x{N}x{K} tA={tA} tB={tB}: max error / bound {ratio.max():.3e}, "
          f"max relative to |A||B| {np.max(np.abs(got - want) / (np.abs(opA) @ np.abs(opB))):.2e}")
    assert np.all(np.isfinite(got))
    assert ratio.max() <= 1.0


def test_tc_gemm_rejects_bad_arguments(ctx):
    import paper_2406_17823_b300 as P
    from ctypes import c_void_p
    lib = P.lib()
    z = c_void_p(0)
    assert lib.qtt_gemm_tf32x3(ctx.h, 0, 4, 4, z, 4, 0, z, 4, 0, z, 4) == 1
    assert lib.qtt_gemm_tf32x3(ctx.h, 4, 4, 4, None, 4, 0, None, 4, 0, None, 4) == 1
    assert lib.qtt_gemm_tf32x3(None, 4, 4, 4, z, 4, 0, z, 4, 0, z, 4) == 1
