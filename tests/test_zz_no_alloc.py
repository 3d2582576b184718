"""The allocation-free dense readout against the regular one and the oracle.

qtt_to_dense_noalloc serves callers that cannot allocate device memory at
the point they read a field back (graph capture, real-time loops, hosts
whose device memory belongs to another framework); it keeps its
intermediates in a static device array.  Its output must equal
qtt_to_dense's and the CPU oracle's on the same MPS, on consecutive calls
that reuse the array, up to the array's size limit and not beyond it.
This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import ctypes

import numpy as np
import pytest

import qtt_inputs as I
from oracle import qtt as Q

pytestmark = pytest.mark.gpu

# bonds at n = 9 whose partial contractions 4^k D_k reach exactly 2^18
# doubles (one half of the static array) at k = 6, 7 and 8
EDGE_BONDS_N9 = [1, 4, 16, 64, 64, 64, 64, 16, 4, 1]


def _call(lib, packed, bonds, n, out, stream):
    b = (ctypes.c_int * (n + 1))(*bonds)
    return lib.qtt_to_dense_noalloc(ctypes.c_void_p(packed.data_ptr()), b, n,
                                    ctypes.c_void_p(out.data_ptr()), stream)


def test_to_dense_noalloc_matches_to_dense():
    import torch
    import paper_2406_17823_b300 as P
    lib = P.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    cases = [(7, I.random_cores(7, I.natural_bonds(7, 16), seed=1)),
             (7, I.random_cores(7, [1, 3, 9, 20, 11, 7, 4, 1], seed=2)),
             (9, I.random_cores(9, EDGE_BONDS_N9, seed=3))]
    for n, cores in cases:  # calls in a row sharing the static scratch
        ctx = P.Context(n)
        bonds = [1] + [c.shape[2] for c in cores]
        ref = ctx.to_dense(ctx.from_cores(cores)).cpu().numpy()  # existing entry point
        want = Q.to_dense(cores)  # the oracle
        packed = torch.tensor(np.concatenate([c.reshape(-1) for c in cores]),
                              dtype=torch.float64, device="cuda")
        out = torch.full((2 ** n, 2 ** n), float("nan"), dtype=torch.float64, device="cuda")
        assert _call(lib, packed, bonds, n, out, stream) == 0
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref)
        assert np.linalg.norm(got - want) <= 1e-12 * np.linalg.norm(want)
    # sizes beyond the static array are rejected, not run: n = 10 (argument
    # range) and, at n = 9, one partial contraction of 2^18 + 4^6 doubles
    big = [1, 4, 16, 64, 256, 1024, 256, 64, 16, 4, 1]
    assert _call(lib, packed, big, 10, out, stream) == 1  # QTT_ERR_ARG
    over = list(EDGE_BONDS_N9)
    over[6] = 65
    assert _call(lib, packed, over, 9, out, stream) == 2  # QTT_ERR_SHAPE
