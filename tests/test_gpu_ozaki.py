"""The mixed form's FP64 product on the BF16 tensor cores (Ozaki splitting,
qtt_gemm_ozaki) against

* a replica of the splitting in exact integer arithmetic, written here from
  the scheme's definition: K taken in chunks of 64; in each chunk every row
  of op(A) (column of op(B)) scaled by 2^e with e the smallest exponent such
  that every |x| < 2^e, the fixed-point value floor(|x| 2^(56 - e)) cut into
  eight 7-bit digits with the sign of x, the digit products of pairs (p, q)
  with p + q <= 7 summed exactly and the exact sum rounded once to the
  nearest FP64 (ties to even); the chunks' results summed in order in FP64.
  The kernel must match it bit for bit: that checks the tensor-core
  accumulation is exact and the integer epilogue rounds correctly;
* the FP64 product, within the scheme's error bound K 2^-53 2^(eA_i + eB_j)
  (eA, eB over the whole K) plus FP64 rounding of the sums.

Shapes: both operand orientations of the kernel (the 128-row side on op(A)
or on op(B)), every output-tile width (16, 32, 64), one and two K chunks,
ragged tiles, batches, several K chunks, alpha and beta, rows of very different scale, zero
rows, and a NaN that must reach exactly its row of the output.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2406_17823_b300 as P
    return P.Context(6)


def scales(X):
    """Per-row scale exponents and Inf/NaN flags of X (rows x K)."""
    mx = (X.view(np.uint64) & np.uint64(0x7FFFFFFFFFFFFFFF)).max(axis=1)
    bad = mx >= np.uint64(0x7FF0000000000000)
    ex = (mx >> np.uint64(52)).astype(np.int64)
    return np.maximum(ex, 1) - 1022, bad


def digits(X, e):
    F = np.floor(np.ldexp(np.abs(np.nan_to_num(X)), (56 - e)[:, None])).astype(np.int64)
    sgn = np.where(np.signbit(X), -1, 1)
    return [sgn * ((F >> (7 * (7 - p))) & 127) for p in range(8)]


def chunk_product(opA, opBt):
    """One K chunk's exact digit products, rounded once to FP64."""
    ea, bada = scales(opA)
    eb, badb = scales(opBt)
    da, db = digits(opA, ea), digits(opBt, eb)
    D = [sum(da[p] @ db[d - p].T for p in range(d + 1)) for d in range(8)]
    assert max(np.abs(x).max() for x in D) < 2 ** 24
    H = ((D[0] * 2 ** 21 + D[1] * 2 ** 14) + D[2] * 2 ** 7) + D[3]
    L = ((D[4] * 2 ** 21 + D[5] * 2 ** 14) + D[6] * 2 ** 7) + D[7]
    sc = ea[:, None] + eb[None, :] - 63
    out = np.empty(H.shape)
    for (i, j), h in np.ndenumerate(H):
        out[i, j] = math.ldexp(float((int(h) << 28) + int(L[i, j])), int(sc[i, j]))
    out[bada, :] = math.nan
    out[:, badb] = math.nan
    return out


def plan(M, N, K, nb, beta=0.0):
    """The kernel's launch plan: the K chunks per slice and the slice count
    (an unbatched product whose 128 x BN output tiles cannot fill the GPU
    deals its chunks over up to 16 slices, at most 16 chunks each)."""
    def bn(r):
        return 64 if r > 32 else 32 if r > 16 else 16

    def padded(ra, rb):
        return -(-ra // 128) * 128 * (-(-rb // bn(rb)) * bn(rb))

    ra, rb = (N, M) if padded(N, M) < padded(M, N) else (M, N)
    tiles = -(-ra // 128) * -(-rb // bn(rb))
    nch = -(-K // 64)
    if nb > 1 or nch == 1:
        return nch, 1
    want = 16 if beta != 0.0 else -(-148 // tiles) if tiles < 74 else 1
    S = max(-(-nch // 16), min(want, min(16, nch)))
    cps = -(-nch // S)
    return cps, -(-nch // cps)


def replica(opA, opBt, alpha, beta, C0, nb=2):
    """K in chunks of 64, each chunk's product with its own scales; within
    a slice the chunk results summed in order in FP64, the slices (if the
    plan splits K) summed in order; then alpha and beta as the kernel (one
    slice) or the slice sum (several) applies them."""
    K = opA.shape[1]
    cps, S = plan(opA.shape[0], opBt.shape[0], K, nb, beta)
    parts = []
    for s0 in range(0, K, 64 * cps):
        acc = None
        for k0 in range(s0, min(K, s0 + 64 * cps), 64):
            x = chunk_product(opA[:, k0:k0 + 64], opBt[:, k0:k0 + 64])
            acc = x if acc is None else acc + x
        parts.append(acc)
    assert len(parts) == S
    if S == 1:
        v = parts[0] if alpha == 1.0 else alpha * parts[0]
        if beta != 0.0:
            v = v + beta * C0  # beta is 0 or 1 here: one rounding, as the kernel's fma
        return v, scales(opA)[0], scales(opBt)[0]
    v = 0.0
    for x in parts:
        v = v + x
    v = alpha * v if beta == 0.0 else alpha * v + beta * C0  # alpha 1, beta 1 here
    return v, scales(opA)[0], scales(opBt)[0]


CASES = [
    # M, N, K, transA, transB, batch, alpha, beta
    (300, 70, 64, False, False, 2, 1.0, 1.0),
    (64, 300, 32, True, False, 4, 1.0, 0.0),
    (200, 48, 128, False, True, 2, -0.5, 0.0),
    (33, 20, 100, True, True, 40, 1.0, 0.0),
    (130, 17, 16, False, False, 64, 0.3, 0.0),
    (96, 24, 65, True, False, 16, -2.0, 0.0),
    (64, 1000, 256, True, False, 2, 1.0, 0.0),
    (256, 64, 768, False, True, 3, 1.0, 0.0),
    # unbatched with few output tiles: K split over 12, 8 and 16 slices
    (256, 64, 768, False, True, 1, 1.0, 1.0),
    (1000, 40, 512, False, False, 1, -0.5, 0.0),
    (64, 200, 4000, True, False, 1, 1.0, 0.0),
    # unbatched, enough tiles: one CTA adds up three chunks in its output
    (9600, 40, 130, False, False, 1, 0.5, 0.0),
    # output tiles 16 wide
    (300, 12, 40, False, False, 64, 1.0, 1.0),
]


@pytest.mark.parametrize("M,N,K,tA,tB,nb,alpha,beta", CASES)
def test_ozaki_matches_replica_and_fp64(ctx, M, N, K, tA, tB, nb, alpha, beta):
    import torch
    rng = np.random.default_rng(M * 131 + N * 7 + K)
    A = rng.standard_normal((nb,) + ((K, M) if tA else (M, K)))
    B = rng.standard_normal((nb,) + ((N, K) if tB else (K, N)))
    # rows of op(A) over six decades, K graded over eight, a zero row
    if tA:
        A *= np.logspace(0, 6, M)[None, None, :] * np.logspace(0, -8, K)[None, :, None]
        A[:, :, 1] = 0.0
    else:
        A *= np.logspace(0, 6, M)[None, :, None] * np.logspace(0, -8, K)[None, None, :]
        A[:, 1, :] = 0.0
    B *= np.logspace(-3, 3, N)[None, None, :] if not tB else np.logspace(-3, 3, N)[None, :, None]
    C0 = rng.standard_normal((nb, M, N))
    opA = np.swapaxes(A, 1, 2) if tA else A
    opB = np.swapaxes(B, 1, 2) if tB else B
    dA, dB = torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda")
    dC = torch.tensor(C0, device="cuda")
    got = ctx.gemm_ozaki(dA, dB, transA=tA, transB=tB, C=dC, alpha=alpha, beta=beta).cpu().numpy()
    worst = 0.0
    for z in range(nb):
        want, ea, eb = replica(opA[z], np.swapaxes(opB[z], 0, 1), alpha, beta, C0[z], nb)
        assert np.array_equal(got[z], want), f"batch {z}: differs from the exact replica"
        exact = alpha * (opA[z] @ opB[z]) + beta * C0[z]
        bound = abs(alpha) * (K * 2.0 ** -53 * np.ldexp(1.0, ea[:, None] + eb[None, :])
                              + K * 2.0 ** -53 * (np.abs(opA[z]) @ np.abs(opB[z]))) \
            + 4 * 2.0 ** -53 * np.abs(exact) + 1e-300
        worst = max(worst, float((np.abs(got[z] - exact) / bound).max()))
    print(f"{M}x{N}x{K} tA={tA} tB={tB} batch {nb}: error / bound {worst:.3f}")
    assert worst <= 1.0


def test_ozaki_nan_reaches_its_row_only(ctx):
    import torch
    rng = np.random.default_rng(5)
    A = rng.standard_normal((256, 64))
    B = rng.standard_normal((64, 160))
    A[7, 3] = np.nan
    got = ctx.gemm_ozaki(torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda")).cpu().numpy()
    assert np.all(np.isnan(got[7]))
    rest = np.delete(got, 7, axis=0)
    assert np.all(np.isfinite(rest))
    want, _, _ = replica(np.delete(A, 7, axis=0), B.T.copy(), 1.0, 0.0, None, nb=1)
    assert np.array_equal(rest, want)


def test_ozaki_rejects_other_shapes(ctx):
    import torch
    import paper_2406_17823_b300 as P
    A = torch.zeros((256, 8), dtype=torch.float64, device="cuda")
    B = torch.zeros((8, 256), dtype=torch.float64, device="cuda")
    with pytest.raises(P.QttError) as e:  # K = 8 < 16
        ctx.gemm_ozaki(A, B)
    assert e.value.status == 2
    A = torch.zeros((2, 256, 1100), dtype=torch.float64, device="cuda")
    B = torch.zeros((2, 1100, 256), dtype=torch.float64, device="cuda")
    with pytest.raises(P.QttError) as e:  # batched, K = 1100 > 1024
        ctx.gemm_ozaki(A, B)
    assert e.value.status == 2
    A = torch.zeros((4, 256, 100), dtype=torch.float64, device="cuda")
    B = torch.zeros((4, 100, 256), dtype=torch.float64, device="cuda")
    with pytest.raises(P.QttError) as e:  # batched, two K chunks and beta != 0
        ctx.gemm_ozaki(A, B, C=torch.zeros((4, 256, 256), dtype=torch.float64, device="cuda"),
                       beta=1.0)
    assert e.value.status == 2


def test_ozaki_projection_shape(ctx):
    """The projection's dominant product at the bench workload (12288 x 256 x
    64: one K chunk, 384 output tiles): 48 sampled rows bit for bit against
    the replica (a row's scale depends on that row only), every element
    within the error bound."""
    import torch
    M, N, K = 12288, 256, 64
    rng = np.random.default_rng(12288)
    A = rng.standard_normal((M, K)) * np.logspace(0, -8, K)[None, :]
    B = rng.standard_normal((K, N)) * np.logspace(-2, 2, N)[None, :]
    got = ctx.gemm_ozaki(torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda")).cpu().numpy()
    rows = np.sort(rng.choice(M, 48, replace=False))
    want, _, _ = replica(A[rows], B.T.copy(), 1.0, 0.0, None, nb=1)
    assert np.array_equal(got[rows], want)
    ea, _ = scales(A)
    eb, _ = scales(B.T.copy())
    exact = A @ B
    bound = K * 2.0 ** -53 * (np.ldexp(1.0, ea[:, None] + eb[None, :]) + np.abs(A) @ np.abs(B)) \
        + 4 * 2.0 ** -53 * np.abs(exact) + 1e-300
    assert float((np.abs(got - exact) / bound).max()) <= 1.0



def test_ozaki_long_k_piece(ctx):
    """The largest single product one launch takes (K = 16384, here 512 x 128:
    the pieces of the chi = 128 environment contractions, K = 3 chi^2 split
    in 16384s): 256 K chunks over 16 K slices summed in order; 6 sampled rows
    bit for bit against the replica, every element within the error bound."""
    import torch
    M, N, K = 512, 128, 16384
    rng = np.random.default_rng(16384)
    A = rng.standard_normal((M, K)) * np.logspace(0, -6, K)[None, :]
    B = rng.standard_normal((K, N))
    got = ctx.gemm_ozaki(torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda")).cpu().numpy()
    rows = np.sort(rng.choice(M, 6, replace=False))
    want, _, _ = replica(A[rows], B.T.copy(), 1.0, 0.0, None, nb=1)
    assert np.array_equal(got[rows], want)
    ea, _ = scales(A)
    eb, _ = scales(B.T.copy())
    exact = A @ B
    bound = K * 2.0 ** -53 * (np.ldexp(1.0, ea[:, None] + eb[None, :]) + np.abs(A) @ np.abs(B)) \
        + 4 * 2.0 ** -53 * np.abs(exact) + 1e-300
    assert float((np.abs(got - exact) / bound).max()) <= 1.0
