"""Mixed-precision form against the FP64 oracle (and the FP64 GPU path).

In the mixed form the SVDs search the kept subspace in FP32; the factor
that becomes the core is re-orthonormalised by an FP64 Householder QR and
the other factor is recomputed as an FP64 projection.  The bar is 1e-6
relative L2 on dense fields.  Bond dimensions may differ from the oracle's
where a rank decision sits at the FP32 noise level, so only fields are
compared.  Sizes are chosen so that the FP32 cluster path is engaged
(square factors of at least 24).
"""
import math

import numpy as np
import pytest

import qtt_inputs as I
from oracle import qtt as Q

pytestmark = pytest.mark.gpu
TOL = 1e-6


def rel(a, b):
    r = float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
    print(f"relative L2 error {r:.3e}")
    return r


@pytest.fixture(scope="module")
def P():
    import paper_2406_17823_b300 as P
    return P


def dense(ctx, m):
    return ctx.to_dense(m).cpu().numpy()


def test_mixed_compress(P):
    n = 6
    ctx = P.Context(n, precision=P.PREC_MIXED)
    A = I.random_cores(n, [1, 4, 16, 48, 16, 4, 1], seed=5)
    A[3] = A[3] * np.logspace(0, -6, 16)[None, None, :]
    for eps, chi in [(1e-8, 64), (0.0, 24)]:
        g = ctx.compress(ctx.from_cores(A), eps, chi)
        o = Q.compress(A, eps, chi)
        assert rel(dense(ctx, g), Q.to_dense(o)) < TOL


def test_mixed_apply_and_hadamard(P):
    n = 7
    X1, X2, dx = I.grid(n)
    ctx = P.Context(n, precision=P.PREC_MIXED)
    ops = Q.build_operators(n, dx)
    F = I.random_field(n, seed=60) + 0.05 * I.white_field(n, seed=61)
    G = I.random_field(n, seed=62) + 0.02 * I.white_field(n, seed=63)
    A, B = Q.from_dense(F, 1e-10, 32), Q.from_dense(G, 1e-10, 32)
    ga, gb = ctx.from_cores(A), ctx.from_cores(B)
    assert rel(dense(ctx, ctx.apply_mpo(1, ga, 1e-10, 32)),
               Q.to_dense(Q.apply_mpo(ops.D[0], A, 1e-10, 32))) < TOL
    assert rel(dense(ctx, ctx.hadamard(ga, gb, 1e-10, 32)),
               Q.to_dense(Q.hadamard(A, B, 1e-10, 32))) < TOL
    assert rel(dense(ctx, ctx.add([1.0, -0.5], [ga, gb], 1e-10, 32)),
               Q.to_dense(Q.add([1.0, -0.5], [A, B], 1e-10, 32))) < TOL


def test_mixed_rk4_jet(P):
    """Shear jet on 2^7 x 2^7 at chi 32, one RK4 step, paper solver settings."""
    n = 7
    u, dx = I.shear_jet(n, delta=2 * math.pi / 60, seed=0)
    dt = 0.1 * dx / np.abs(u[0]).max()
    pp = dict(eps=1e-8, chi_max=32)
    ctx = P.Context(n, precision=P.PREC_MIXED, **pp)
    p = Q.Params(**pp)
    ops = Q.build_operators(n, dx)
    uq = [Q.from_dense(f, p.eps, p.chi_max) for f in u]
    g = [ctx.from_cores(c) for c in uq]
    ref = Q.rk4_step(uq, dt, 1 / 2e5, p, ops)
    ctx.rk4_step(g[0], g[1], dt, 1 / 2e5)
    for i in range(2):
        assert rel(dense(ctx, g[i]), Q.to_dense(ref[i])) < TOL


def test_mixed_matches_fp64_at_full_size(P):
    """The benchmark configuration (2^10 x 2^10 shear jet, chi 64, paper
    settings): one mixed RK4 step against the FP64 GPU step, which the
    parity suite ties to the oracle."""
    import qtt_inputs as I2
    n = 10
    u, dx = I2.shear_jet(n, seed=0)
    dt = 0.1 * dx / np.abs(u[0]).max()
    f64 = P.Context(n, eps=1e-8, chi_max=64)
    mix = P.Context(n, eps=1e-8, chi_max=64, precision=P.PREC_MIXED)
    g64 = [f64.from_dense(f) for f in u]
    cores = [f64.to_cores(x) for x in g64]
    gmx = [mix.from_cores(c) for c in cores]
    f64.rk4_step(g64[0], g64[1], dt, 1 / 2e5)
    mix.rk4_step(gmx[0], gmx[1], dt, 1 / 2e5)
    for i in range(2):
        assert rel(dense(mix, gmx[i]), dense(f64, g64[i])) < TOL


def test_mixed_stays_within_bar_over_steps(P):
    """Six RK4 steps, mixed against FP64 on the GPU (2^7 jet, chi 64, which
    is the natural bound there): the per-cut error of the FP32 subspace
    search is shrunk by one FP64 subspace iteration, so the difference does
    not build up past the bar."""
    n = 7
    u, dx = I.shear_jet(n, seed=0)
    dt = 0.1 * dx / np.abs(u[0]).max()
    f64 = P.Context(n, eps=1e-8, chi_max=64)
    mix = P.Context(n, eps=1e-8, chi_max=64, precision=P.PREC_MIXED)
    gf = [f64.from_dense(f) for f in u]
    gm = [mix.from_cores(f64.to_cores(x)) for x in gf]
    errs = []
    for _ in range(6):
        f64.rk4_step(gf[0], gf[1], dt, 1 / 2e5)
        mix.rk4_step(gm[0], gm[1], dt, 1 / 2e5)
        errs.append(max(rel(dense(mix, gm[i]), dense(f64, gf[i])) for i in range(2)))
    print("mixed vs FP64 after 1..6 steps:", ["%.1e" % e for e in errs])
    assert max(errs) < TOL
