"""The paper's form of the step (Sec. II.C, App. B; qtt_params.rhs_form =
QTT_RHS_IMPLICIT) on the GPU against the oracle's: each stage's right-hand
side a u - h B(b) is never formed -- its Hadamard products and MPO terms are
contracted inside the projection's environments (the nonlinear terms as
products of a Hadamard MPO and D_j), and the initial guess is a u.  Dense
fields within 1e-10 (FP64) and 1e-6 (mixed) of the oracle's
rk4_step_implicit; at full rank
also equal to the dense projected RK4 step; whole-step graphs replay it bit
for bit.
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


def test_implicit_rk4_full_rank_equals_dense(P):
    n = 4
    X1, X2, dx = I.grid(n)
    u0, _ = I.taylor_green(n)
    u = [u0[0] + 0.1 * I.random_field(n, seed=3), u0[1] + 0.1 * I.random_field(n, seed=4)]
    tight = dict(eps=0.0, chi_max=256, cg_tol=1e-13, cg_maxit=500, sweep_tol=1e-13,
                 max_sweeps=40)
    ctx = P.Context(n, rhs_form=P.RHS_IMPLICIT, **tight)
    g = [ctx.from_dense(f, 0.0, 256) for f in u]
    ctx.rk4_step(g[0], g[1], 1e-2, 0.01)
    ref = Dn.rk4_step(u, 1e-2, 0.01, 2.5e5, dx)
    for i in range(2):
        assert rel(ctx.to_dense(g[i]).cpu().numpy(), ref[i]) <= TOL


@pytest.mark.parametrize("prec,tol", [(0, TOL), (1, 1e-6)])
@pytest.mark.parametrize("n,chi", [(6, 16), (7, 32)])
def test_implicit_rk4_matches_oracle(P, n, chi, prec, tol):
    """Shear jet, paper solver settings, truncated (eps 1e-8, chi cap); the
    FP64 form at 1e-10, the mixed form (its products on the tensor cores by
    the Ozaki splitting, its cuts by the tensor-core search) at 1e-6."""
    (u, v), dx = I.shear_jet(n, delta=2 * math.pi / 60, seed=0)
    dt, nu = 0.1 * dx / float(np.abs(u).max()), 1 / 2e5
    pp = dict(eps=1e-8, chi_max=chi)
    ctx = P.Context(n, rhs_form=P.RHS_IMPLICIT, precision=prec, **pp)
    uq = [Q.from_dense(f, pp["eps"], chi) for f in (u, v)]
    g = [ctx.from_cores(c) for c in uq]
    ref = Q.rk4_step_implicit(uq, dt, nu, Q.Params(**pp), Q.build_operators(n, dx))
    ctx.rk4_step(g[0], g[1], dt, nu)
    for i in range(2):
        assert rel(ctx.to_dense(g[i]).cpu().numpy(), Q.to_dense(ref[i])) <= tol


@pytest.mark.parametrize("prec", [0, 1])
def test_implicit_step_graph_replays_bit_for_bit(P, prec):
    (u, v), dx = I.shear_jet(6, seed=2)
    dt, nu = 0.1 * dx / float(np.abs(u).max()), 1e-4
    out = []
    for graphs in (0, 2):
        ctx = P.Context(6, eps=1e-8, chi_max=16, graphs=graphs, rhs_form=P.RHS_IMPLICIT,
                        precision=prec)
        a, b = ctx.from_dense(u), ctx.from_dense(v)
        for _ in range(4):
            ctx.rk4_step(a, b, dt, nu)
        if graphs:
            assert ctx.graph_stats()[1] >= 2
        out.append([ctx.to_dense(a).cpu().numpy(), ctx.to_dense(b).cpu().numpy()])
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_forms_at_equal_error_full_size(P):
    """The bench workload (2^10 jet, chi 64, eps 1e-8, paper settings): one
    RK4 step in each form against the untruncated dense projected RK4 step
    from the same (truncated) initial state.  Both forms carry the same
    truncation error (printed); the implicit one may not exceed the explicit
    one's by more than half."""
    n = 10
    (u, v), dx = I.shear_jet(n, seed=0)
    dt, nu = 0.1 * dx / float(np.abs(u).max()), 1 / 2e5
    errs = {}
    for form in (P.RHS_EXPLICIT, P.RHS_IMPLICIT):
        ctx = P.Context(n, eps=1e-8, chi_max=64, rhs_form=form)
        g = [ctx.from_dense(f) for f in (u, v)]
        u0 = [ctx.to_dense(x).cpu().numpy() for x in g]
        ref = Dn.rk4_step(u0, dt, nu, 2.5e5, dx)
        ctx.rk4_step(g[0], g[1], dt, nu)
        got = [ctx.to_dense(x).cpu().numpy() for x in g]
        num = sum(float(np.sum((a - b) ** 2)) for a, b in zip(got, ref))
        den = sum(float(np.sum(b ** 2)) for b in ref)
        errs[form] = math.sqrt(num / den)
    print(f"one RK4 step vs the dense step: explicit {errs[0]:.3e}, implicit {errs[1]:.3e}")
    assert errs[1] <= 1.5 * errs[0] + 1e-14


@pytest.fixture(scope="module")
def implicit_full_ref():
    """The oracle's implicit RK4 step on the bench workload (2^10 shear jet,
    chi 64, eps 1e-8, the paper's solver settings): about a minute on one
    core."""
    n = 10
    (u, v), dx = I.shear_jet(n, seed=0)
    dt, nu = 0.1 * dx / float(np.abs(u).max()), 1 / 2e5
    pp = dict(eps=1e-8, chi_max=64)
    uq = [Q.from_dense(f, pp["eps"], pp["chi_max"]) for f in (u, v)]
    ref = Q.rk4_step_implicit(uq, dt, nu, Q.Params(**pp), Q.build_operators(n, dx))
    return n, uq, dt, nu, [Q.to_dense(r) for r in ref]


@pytest.mark.parametrize("prec,tol", [(0, TOL), (1, 1e-6)])
def test_implicit_full_size_matches_oracle(P, implicit_full_ref, prec, tol):
    """One RK4 step of the bench's headline scheme at full size, replayed as a
    whole-step graph where the bench replays it: FP64 within 1e-10, mixed
    (products on the tensor cores) within 1e-6 of the oracle's step."""
    n, uq, dt, nu, want = implicit_full_ref
    ctx = P.Context(n, eps=1e-8, chi_max=64, rhs_form=P.RHS_IMPLICIT, precision=prec, graphs=2)
    g = [ctx.from_cores(c) for c in uq]
    ctx.rk4_step(g[0], g[1], dt, nu)
    for i in range(2):
        assert rel(ctx.to_dense(g[i]).cpu().numpy(), want[i]) <= tol
