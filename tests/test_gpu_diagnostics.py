"""Diagnostics on the GPU: the MPS inner product against the oracle's
transfer matrices, and the closed forms it must reproduce (the Taylor-Green
kinetic energy 1/4, the fidelity of a state with itself and with a scaled
copy)."""
import numpy as np
import pytest

import qtt_inputs as I
from oracle import qtt as Q

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2406_17823_b300 as P
    return P


def test_inner_matches_oracle(P):
    n = 6
    ctx = P.Context(n)
    A = I.random_cores(n, [1, 4, 16, 33, 16, 4, 1], seed=11)
    B = I.random_cores(n, [1, 3, 9, 20, 12, 4, 1], seed=12)
    got = ctx.inner(ctx.from_cores(A), ctx.from_cores(B))
    want = Q.inner(A, B)
    assert abs(got - want) <= 1e-12 * max(1.0, abs(want))
    # and the dense definition
    dense = float(np.sum(Q.to_dense(A) * Q.to_dense(B)))
    assert abs(got - dense) <= 1e-11 * max(1.0, abs(dense))


def test_taylor_green_energy_and_fidelity(P):
    n = 6
    ctx = P.Context(n)
    (u, v), dx = I.taylor_green(n)
    a, b = ctx.from_dense(u), ctx.from_dense(v)
    assert abs(ctx.kinetic_energy(a, b) - 0.25) < 1e-13
    assert abs(ctx.fidelity(a, a) - 1.0) < 1e-13
    c = ctx.add([-3.0], [a])
    assert abs(ctx.fidelity(a, c) - 1.0) < 1e-13
    assert ctx.fidelity(a, b) < 1e-20  # sin x cos y and cos x sin y are orthogonal
