"""GPU (CUDA library, FP64 path) against the CPU oracle, op by op.

Inputs are identical on both sides: seeded fields / cores from qtt_inputs,
handed to the oracle as numpy arrays and to the library through the C ABI.
Results are compared as dense fields (the gauge of the cores is not
unique) together with the bond dimensions and, for the projection, the CG
iteration and sweep counts (the stopping decisions must coincide).

FP64 tolerance: 1e-10 relative L2 for whole steps (the bar the FP64 path
must meet), tighter for single operations.
"""
import math

import numpy as np
import pytest

import qtt_inputs as I
from oracle import dense as Dn
from oracle import qtt as Q

pytestmark = pytest.mark.gpu

FULL = 10 ** 6


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def Q3():
    import torch
    import paper_2406_17823_b300 as P
    assert torch.cuda.is_available()
    return P


def ctx_for(P, n, **kw):
    return P.Context(n, **kw)


def gpu_dense(ctx, m):
    return ctx.to_dense(m).cpu().numpy()


# ------------------------------------------------------------ encoding
@pytest.mark.parametrize("n", [1, 2, 5, 7])
def test_from_dense_roundtrip_and_bonds(Q3, n):
    ctx = ctx_for(Q3, n)
    F = I.random_field(n, seed=n) + 0.01 * I.white_field(n, seed=n + 1)
    for eps, chi in [(0.0, FULL), (1e-3, FULL), (1e-10, 8)]:
        g = ctx.from_dense(F, eps, chi)
        o = Q.from_dense(F, eps, chi)
        assert g.bonds == Q.bond_dims(o)
        assert rel(gpu_dense(ctx, g), Q.to_dense(o)) < 1e-12


def test_packed_roundtrip(Q3):
    n = 6
    ctx = ctx_for(Q3, n)
    A = I.random_cores(n, [1, 4, 16, 9, 16, 4, 1], seed=3)
    g = ctx.from_cores(A)
    assert g.bonds == Q.bond_dims(A)
    assert rel(gpu_dense(ctx, g), Q.to_dense(A)) < 1e-14
    back = ctx.to_cores(g)
    for a, b in zip(A, back):
        np.testing.assert_array_equal(a, b)


# ------------------------------------------------------------ single ops
@pytest.mark.parametrize("eps,chi", [(0.0, FULL), (1e-6, FULL), (0.0, 7), (1e-2, 5)])
def test_compress_parity(Q3, eps, chi):
    n = 6
    ctx = ctx_for(Q3, n)
    A = I.random_cores(n, [1, 4, 16, 30, 16, 4, 1], seed=11)
    # make the spectrum decay so that eps matters
    A[3] = A[3] * np.linspace(1, 1e-4, A[3].shape[2])[None, None, :]
    g = ctx.compress(ctx.from_cores(A), eps, chi)
    o = Q.compress(A, eps, chi)
    assert g.bonds == Q.bond_dims(o)
    assert rel(gpu_dense(ctx, g), Q.to_dense(o)) < 1e-12


@pytest.mark.parametrize("which", [1, 2, 3])
def test_apply_mpo_parity(Q3, which):
    n = 6
    X1, X2, dx = I.grid(n)
    ctx = ctx_for(Q3, n)
    ops = Q.build_operators(n, dx)
    W = {1: ops.D[0], 2: ops.D[1], 3: ops.lap}[which]
    F = I.random_field(n, seed=21) + 0.05 * I.white_field(n, seed=22)
    A = Q.from_dense(F, 1e-9, 24)
    for eps, chi in [(0.0, FULL), (1e-8, 24)]:
        g = ctx.apply_mpo(which, ctx.from_cores(A), eps, chi)
        o = Q.apply_mpo(W, A, eps, chi)
        assert g.bonds == Q.bond_dims(o)
        assert rel(gpu_dense(ctx, g), Q.to_dense(o)) < 1e-11


def test_projection_operators_match_stencils(Q3):
    """The library's own MPOs (built from the carry table on the host)
    act like the dense stencils, including the D_i^T D_j blocks."""
    n = 5
    X1, X2, dx = I.grid(n)
    ctx = ctx_for(Q3, n)
    F = I.white_field(n, seed=7)
    A = ctx.from_dense(F, 0.0, FULL)
    want = {1: Dn.d(F, 1, dx), 2: Dn.d(F, 2, dx),
            3: sum(Dn.d(Dn.d(F, j, dx), j, dx) for j in (1, 2))}
    for i in range(2):
        for j in range(2):
            want[4 + 2 * i + j] = -Dn.d(Dn.d(F, j + 1, dx), i + 1, dx)
    for which, w in want.items():
        g = ctx.apply_mpo(which, A, 0.0, FULL)
        assert rel(gpu_dense(ctx, g), w) < 1e-12, which


@pytest.mark.parametrize("k", [1, 2, 3])
def test_add_parity(Q3, k):
    n = 5
    ctx = ctx_for(Q3, n)
    terms = [I.random_cores(n, [1, 4, 6 + t, 5, 4, 1], seed=30 + t) for t in range(k)]
    coefs = [0.5, -1.25, 2.0][:k]
    g = ctx.add(coefs, [ctx.from_cores(t) for t in terms], 1e-9, 12)
    o = Q.add(coefs, terms, 1e-9, 12)
    assert g.bonds == Q.bond_dims(o)
    assert rel(gpu_dense(ctx, g), Q.to_dense(o)) < 1e-12


@pytest.mark.parametrize("chi", [4, 9, 64])
def test_hadamard_parity(Q3, chi):
    n = 6
    ctx = ctx_for(Q3, n)
    F = I.random_field(n, seed=40) + 0.1 * I.white_field(n, seed=41)
    G = I.random_field(n, seed=42)
    A, B = Q.from_dense(F, 1e-6, 10), Q.from_dense(G, 1e-10, 10)
    g = ctx.hadamard(ctx.from_cores(A), ctx.from_cores(B), 1e-10, chi)
    o = Q.hadamard(A, B, 1e-10, chi)
    assert g.bonds == Q.bond_dims(o)
    assert rel(gpu_dense(ctx, g), Q.to_dense(o)) < 1e-11


def test_zero_and_degenerate_inputs(Q3):
    n = 4
    ctx = ctx_for(Q3, n)
    Z = [np.zeros((b0, 4, b1)) for b0, b1 in zip([1, 4, 8, 4], [4, 8, 4, 1])]
    z = ctx.compress(ctx.from_cores(Z), 1e-8, 8)
    assert z.bonds == Q.bond_dims(Q.compress(Z, 1e-8, 8))
    assert np.all(gpu_dense(ctx, z) == 0.0)
    h = ctx.hadamard(z, z, 1e-8, 8)
    assert np.all(gpu_dense(ctx, h) == 0.0)
    # a field constant along x1 has a zero x1-derivative
    X1, X2, dx = I.grid(n)
    c = ctx.from_dense(np.cos(X2), 1e-12, 8)
    d1 = ctx.apply_mpo(1, c, 1e-12, 8)
    assert np.abs(gpu_dense(ctx, d1)).max() < 1e-12


# ------------------------------------------------------------ projection
@pytest.mark.parametrize("h,full", [(1e-3, True), (1e-2, True), (2e-3, False)])
def test_projection_parity(Q3, h, full):
    n = 5
    ctx = ctx_for(Q3, n, cg_tol=1e-12, cg_maxit=500, sweep_tol=1e-12, max_sweeps=30)
    X1, X2, dx = I.grid(n)
    ops = Q.build_operators(n, dx)
    if full:
        w = [I.white_field(n, seed=50), I.white_field(n, seed=51)]
        wq = [Q.from_dense(f, 0.0, FULL) for f in w]
    else:
        w = [I.random_field(n, seed=52) + 0.01 * I.white_field(n, seed=53),
             I.random_field(n, seed=54)]
        wq = [Q.from_dense(f, 1e-6, 6) for f in w]
    p = Q.Params(eps=0.0, chi_max=FULL, cg_tol=1e-12, cg_maxit=500, sweep_tol=1e-12, max_sweeps=30)
    vo, info = Q.project(wq, h, p, ops)
    v1, v2, cg, sw, ok = ctx.project(ctx.from_cores(wq[0]), ctx.from_cores(wq[1]), h)
    assert sw == info.sweeps
    assert abs(cg - info.cg_iters) <= max(2, info.cg_iters // 100)
    for g, o in zip((v1, v2), vo):
        assert rel(gpu_dense(ctx, g), Q.to_dense(o)) < 1e-10
    if full:
        vd = Dn.project(w, h, p.mu, dx)
        assert rel(gpu_dense(ctx, v1), vd[0]) < 1e-9


def test_projection_mu_argument(Q3):
    """qtt_project's own penalty (mu = 1e3 on a context made with the
    paper's 2.5e5) against the oracle's projection with that mu."""
    n, h = 5, 1e-2
    ctx = ctx_for(Q3, n, cg_tol=1e-12, cg_maxit=500, sweep_tol=1e-12, max_sweeps=30)
    X1, X2, dx = I.grid(n)
    ops = Q.build_operators(n, dx)
    w = [I.white_field(n, seed=55), I.white_field(n, seed=56)]
    wq = [Q.from_dense(f, 0.0, FULL) for f in w]
    p = Q.Params(eps=0.0, chi_max=FULL, mu=1e3, cg_tol=1e-12, cg_maxit=500, sweep_tol=1e-12,
                 max_sweeps=30)
    vo, info = Q.project(wq, h, p, ops)
    v1, v2, cg, sw, ok = ctx.project(ctx.from_cores(wq[0]), ctx.from_cores(wq[1]), h, mu=1e3)
    for g, o in zip((v1, v2), vo):
        assert rel(gpu_dense(ctx, g), Q.to_dense(o)) < 1e-10
    vd = Dn.project(w, h, 1e3, dx)
    assert rel(gpu_dense(ctx, v1), vd[0]) < 1e-9


# ------------------------------------------------------------ RK4 step
def _rk4_case(Q3, n, u, dt, nu, steps, **pp):
    ctx = ctx_for(Q3, n, **pp)
    X1, X2, dx = I.grid(n)
    ops = Q.build_operators(n, dx)
    p = Q.Params(**pp)
    uq = [Q.from_dense(f, p.eps, p.chi_max) for f in u]
    g = [ctx.from_cores(c) for c in uq]
    for _ in range(steps):
        uq = Q.rk4_step(uq, dt, nu, p, ops)
        ctx.rk4_step(g[0], g[1], dt, nu)
    for i in range(2):
        assert g[i].bonds == Q.bond_dims(uq[i])
        assert rel(gpu_dense(ctx, g[i]), Q.to_dense(uq[i])) < 1e-10
    return ctx, g, uq


def test_rk4_taylor_green_parity(Q3):
    """Taylor-Green, 2^6 x 2^6, chi 16, eps 1e-12, nu 0.01, dt 1e-3."""
    n = 6
    u, dx = I.taylor_green(n)
    _rk4_case(Q3, n, u, 1e-3, 0.01, 2, eps=1e-12, chi_max=16, cg_tol=1e-12, cg_maxit=500,
              sweep_tol=1e-12, max_sweeps=20)


def test_rk4_jet_small_parity(Q3):
    """Shear-jet initial condition on 2^6 x 2^6 at chi 8 (truncation
    active at every bond) with the paper's solver tolerances."""
    n = 6
    u, dx = I.shear_jet(n, delta=2 * math.pi / 40, seed=0)
    dt = 0.1 * dx / np.abs(u[0]).max()
    _rk4_case(Q3, n, u, dt, 1 / 2e5, 1, eps=1e-8, chi_max=8)


def test_error_statuses(Q3):
    n = 4
    ctx = ctx_for(Q3, n)
    F = np.ones((16, 16))
    F[3, 3] = np.nan
    with pytest.raises(Q3.QttError) as e:
        m = ctx.from_dense(F, 1e-8, 8)
        ctx.to_dense(m)
    assert e.value.status == 7
    ok = ctx.from_dense(np.ones((16, 16)), 1e-8, 8)
    ctx.sync()
    with pytest.raises(Q3.QttError) as e:
        ctx.add([1.0] * 9, [ok] * 9)
    assert e.value.status == 1
    ctx5 = ctx_for(Q3, 5)
    other = ctx5.from_dense(np.ones((32, 32)), 1e-8, 8)
    with pytest.raises(Q3.QttError) as e:
        ctx.hadamard(ok, other)
    assert e.value.status == 2
