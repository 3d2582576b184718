"""Bond caps past 64 (the chi = 128 and chi = 256 configurations): factors
wider than 256 columns, which the cluster SVD serves with its scalar
tournament (columns homed in distributed shared memory) instead of the
register-resident systolic kernel, against the oracle.

At n = 9 with chi = 128 the two middle bonds are at the cap: an MPO
application makes 384-wide factors (3 chi), a sum 256-wide ones (2 chi) and
the Hadamard zip-up 512-row factors (4 chi rows, chi^2 columns).  With
chi = 256 the application reaches 768 and the sum 512.  Every result is
compared with the oracle's on the reconstructed dense field: 1e-10 for the
FP64 form, 1e-6 for the mixed form (whose searches fall back to the FP32
cluster SVD at these widths).
"""
import numpy as np
import pytest

import qtt_inputs as I
from oracle import qtt as Q

pytestmark = pytest.mark.gpu
N_BITS, EPS = 9, 1e-10


@pytest.fixture(scope="module")
def fields():
    F = I.random_field(N_BITS, seed=1) + 1e-3 * I.white_field(N_BITS, seed=2)
    G = I.random_field(N_BITS, seed=3) + 1e-3 * I.white_field(N_BITS, seed=4)
    X1, X2, dx = I.grid(N_BITS)
    return F, G, Q.build_operators(N_BITS, dx)


def rel(a, b):
    r = float(np.linalg.norm(a - b) / np.linalg.norm(b))
    print(f"relative L2 {r:.2e}")
    return r


def dense(ctx, m):
    return ctx.to_dense(m).cpu().numpy()


@pytest.mark.parametrize("chi", [128, 256])
@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-6)])
def test_apply_and_add_wide(fields, chi, prec, tol):
    import paper_2406_17823_b300 as P
    F, G, ops = fields
    ctx = P.Context(N_BITS, eps=EPS, chi_max=chi, precision=prec)
    A, B = Q.from_dense(F, EPS, chi), Q.from_dense(G, EPS, chi)
    assert max(Q.bond_dims(A)) == chi  # the cap is reached
    ga, gb = ctx.from_cores(A), ctx.from_cores(B)
    assert rel(dense(ctx, ctx.apply_mpo(1, ga)), Q.to_dense(Q.apply_mpo(ops.D[0], A, EPS, chi))) <= tol
    assert rel(dense(ctx, ctx.apply_mpo(3, gb)), Q.to_dense(Q.apply_mpo(ops.lap, B, EPS, chi))) <= tol
    assert rel(dense(ctx, ctx.add([1.0, -0.7], [ga, gb])),
               Q.to_dense(Q.add([1.0, -0.7], [A, B], EPS, chi))) <= tol


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-6)])
def test_hadamard_chi128(fields, prec, tol):
    import paper_2406_17823_b300 as P
    F, G, ops = fields
    chi = 128
    ctx = P.Context(N_BITS, eps=EPS, chi_max=chi, precision=prec)
    A, B = Q.from_dense(F, EPS, chi), Q.from_dense(G, EPS, chi)
    got = dense(ctx, ctx.hadamard(ctx.from_cores(A), ctx.from_cores(B)))
    assert rel(got, Q.to_dense(Q.hadamard(A, B, EPS, chi))) <= tol


def test_rk4_step_turbulence_chi128():
    """One RK4 step in the shape of the chi = 128 turbulence configuration
    (2^11 x 2^11, seeded random-phase vorticity with E(k) ~ k^4
    exp(-2 (k / 10)^2), unit kinetic energy, eps = 1e-7, chi = 128, Re = 1e6,
    dt = 0.1 dx / max|u|, the paper's solver settings): the step grows the
    first middle bond to the cap.  FP64 form against the oracle at 1e-10,
    mixed form at 1e-6 (about a minute of oracle time)."""
    import paper_2406_17823_b300 as P
    n, chi, eps = 11, 128, 1e-7
    (u, v), dx = I.decaying_turbulence(n, k0=10, seed=0)
    dt = 0.1 * dx / float(max(np.abs(u).max(), np.abs(v).max()))
    nu = 1e-6
    prm = Q.Params(eps=eps, chi_max=chi)
    uq = [Q.from_dense(f, eps, chi) for f in (u, v)]
    ref = Q.rk4_step(uq, dt, nu, prm, Q.build_operators(n, dx))
    assert max(Q.bond_dims(ref[0])) == chi
    want = [Q.to_dense(r) for r in ref]
    for prec, tol in ((0, 1e-10), (1, 1e-6)):
        ctx = P.Context(n, eps=eps, chi_max=chi, precision=prec, graphs=2)
        g = [ctx.from_cores(c) for c in uq]
        ctx.rk4_step(g[0], g[1], dt, nu)
        for got, w in zip(g, want):
            assert rel(dense(ctx, got), w) <= tol


def test_implicit_long_k_products_chi128(fields):
    """The paper's implicit step at chi = 128 (n = 9, middle bonds at the
    cap): its environment contractions have K = 3 chi^2 = 49152, past what
    one emulated launch takes, so the mixed form runs them as K pieces on the
    tensor cores accumulated in order.  Mixed within 1e-10 of the FP64 form
    after one RK4 step (the emulated products are FP64-accurate; the FP64
    implicit form is pinned to the oracle at chi = 16..64)."""
    import paper_2406_17823_b300 as P
    F, G, ops = fields
    chi = 128
    dx = 2 * np.pi / 2 ** N_BITS
    dt, nu = 0.1 * dx / float(max(np.abs(F).max(), np.abs(G).max())), 1e-4
    out = []
    for prec in (0, 1):
        ctx = P.Context(N_BITS, eps=1e-8, chi_max=chi, precision=prec,
                        rhs_form=P.RHS_IMPLICIT)
        g = [ctx.from_cores(Q.from_dense(f, 1e-8, chi)) for f in (F, G)]
        assert max(g[0].bonds) == chi
        ctx.rk4_step(g[0], g[1], dt, nu)
        out.append([dense(ctx, x) for x in g])
    for a, b in zip(out[1], out[0]):
        assert rel(a, b) <= 1e-10
