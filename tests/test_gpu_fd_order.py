"""Higher-order central differences (Sec. II.B: finite-difference
operators of any order; App. D's 8th-order stencil) on the GPU against the
oracle: the derivative and Laplacian MPOs of orders 4, 6 and 8 applied to
seeded fields, qtt_mpo_diff (the C ABI's derivative operator for a caller's
axis, power and spacing) against the oracle's MPO and the dense stencil,
and one RK4 step with 4th-order stencils against the oracle (relative L2
on dense fields, 1e-10, the FP64 bar).
"""
import math

import numpy as np
import pytest

import qtt_inputs as I
from oracle import dense as Dn
from oracle import qtt as Q

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def P():
    import paper_2406_17823_b300 as P
    return P


def rel(a, b):
    r = float(np.linalg.norm(a - b) / np.linalg.norm(b))
    print(f"relative L2 {r:.2e}")
    return r


@pytest.mark.parametrize("order", [4, 6, 8])
def test_apply_high_order_operators(P, order):
    n = 7
    X1, X2, dx = I.grid(n)
    ctx = P.Context(n, eps=1e-12, chi_max=64, fd_order=order)
    ops = Q.build_operators(n, dx, order=order)
    F = I.random_field(n, seed=70 + order) + 0.02 * I.white_field(n, seed=71)
    A = Q.from_dense(F, 1e-12, 64)
    g = ctx.from_cores(A)
    for which, W in ((1, ops.D[0]), (2, ops.D[1]), (3, ops.lap)):
        got = ctx.to_dense(ctx.apply_mpo(which, g)).cpu().numpy()
        want = Q.to_dense(Q.apply_mpo(W, A, 1e-12, 64))
        assert rel(got, want) <= TOL
    # the projection blocks D_i^T D_j through the dense stencil
    f = I.white_field(5, seed=3)
    ctx5 = P.Context(5, fd_order=order)
    dx5 = 2 * math.pi / 32
    q5 = ctx5.from_dense(f, 0.0, 1024)
    for which, (i, j) in ((4, (0, 0)), (5, (0, 1)), (6, (1, 0)), (7, (1, 1))):
        got = ctx5.to_dense(ctx5.apply_mpo(which, q5, 0.0, 1024)).cpu().numpy()
        want = -Dn.d(Dn.d(f, j + 1, dx5, order), i + 1, dx5, order)
        assert rel(got, want) <= 1e-12


@pytest.mark.parametrize("order", [2, 4, 8])
@pytest.mark.parametrize("axis", [1, 2])
@pytest.mark.parametrize("power", [1, 2])
def test_mpo_diff_entry_point(P, order, axis, power):
    """qtt_mpo_diff(axis, power, dx): D or D D of the context's order with
    the caller's spacing, against the dense stencil (here dx = 0.37, not
    the context's L / N)."""
    n = 5
    dx = 0.37
    ctx = P.Context(n, fd_order=order)
    f = I.white_field(n, seed=10 * axis + power)
    q = ctx.from_dense(f, 0.0, 1024)
    m = ctx.mpo_diff(axis, power, dx)
    try:
        got = ctx.to_dense(ctx.apply_mpo(m, q, 0.0, 1024)).cpu().numpy()
    finally:
        ctx.free_mpo(m)
    want = Dn.d(f, axis, dx, order)
    if power == 2:
        want = Dn.d(want, axis, dx, order)
    assert rel(got, want) <= 1e-12


def test_mpo_diff_rejects_bad_arguments(P):
    ctx = P.Context(4)
    with pytest.raises(P.QttError):
        ctx.mpo_diff(3, 1, 0.1)
    with pytest.raises(P.QttError):
        ctx.mpo_diff(1, 3, 0.1)
    with pytest.raises(P.QttError):
        ctx.mpo_diff(1, 1, 0.0)


def test_rk4_step_fourth_order(P):
    """One RK4 step with 4th-order stencils (shear jet 2^7, chi 32, paper
    solver settings) against the oracle's step with the same operators."""
    n = 7
    (u, v), dx = I.shear_jet(n, delta=2 * math.pi / 60, seed=0)
    dt, nu = 0.1 * dx / float(np.abs(u).max()), 1 / 2e5
    pp = dict(eps=1e-8, chi_max=32)
    ctx = P.Context(n, fd_order=4, **pp)
    ops = Q.build_operators(n, dx, order=4)
    uq = [Q.from_dense(f, pp["eps"], pp["chi_max"]) for f in (u, v)]
    g = [ctx.from_cores(c) for c in uq]
    ref = Q.rk4_step(uq, dt, nu, Q.Params(**pp), ops)
    ctx.rk4_step(g[0], g[1], dt, nu)
    for i in range(2):
        assert rel(ctx.to_dense(g[i]).cpu().numpy(), Q.to_dense(ref[i])) <= TOL
