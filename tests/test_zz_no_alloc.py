"""The allocation-free dense readout against the regular one.

qtt_to_dense_noalloc serves callers that cannot allocate device memory at
the point they read a field back (graph capture, real-time loops, hosts
whose device memory belongs to another framework); it keeps its
intermediates in a static device array.  Its output must equal
qtt_to_dense's on the same MPS, on consecutive calls that reuse the array.
This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import ctypes

import numpy as np
import pytest

import qtt_inputs as I

pytestmark = pytest.mark.gpu


def test_to_dense_noalloc_matches_to_dense():
    import torch
    import paper_2406_17823_b300 as P
    lib = P.lib()
    n = 7
    ctx = P.Context(n)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    cases = [I.random_cores(n, I.natural_bonds(n, 16), seed=1),
             I.random_cores(n, [1, 3, 9, 20, 11, 7, 4, 1], seed=2)]
    for cores in cases:  # two calls in a row sharing the static scratch
        bonds = [1] + [c.shape[2] for c in cores]
        ref = ctx.to_dense(ctx.from_cores(cores)).cpu().numpy()  # existing entry point
        packed = torch.tensor(np.concatenate([c.reshape(-1) for c in cores]),
                              dtype=torch.float64, device="cuda")
        out = torch.full((2 ** n, 2 ** n), float("nan"), dtype=torch.float64, device="cuda")
        b = (ctypes.c_int * (n + 1))(*bonds)
        st = lib.qtt_to_dense_noalloc(ctypes.c_void_p(packed.data_ptr()), b, n,
                                      ctypes.c_void_p(out.data_ptr()), stream)
        assert st == 0
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref)
    # sizes beyond the static array are rejected, not run
    big = (ctypes.c_int * 11)(1, 4, 16, 64, 256, 1024, 256, 64, 16, 4, 1)
    assert lib.qtt_to_dense_noalloc(ctypes.c_void_p(packed.data_ptr()), big, 10,
                                    ctypes.c_void_p(out.data_ptr()), stream) != 0
