"""Parity at the bench's full size (2^10 x 2^10, chi = 64, eps = 1e-8).

The step's operations one at a time on the bench workload's own state (the
seeded shear jet): the TT-SVD of the initial field, the derivative and
Laplacian MPO applications, the Hadamard product of the convection term and
a block-diagonal sum; then one whole RK4 step at the bench's settings (about
half a minute of oracle time), with the stage graphs the bench replays.
Each against the FP64 oracle to 1e-10 relative L2 on the reconstructed
dense fields.
"""
import numpy as np
import pytest

import qtt_inputs as I
from oracle import qtt as Q

pytestmark = pytest.mark.gpu
N_BITS, CHI, EPS, TOL = 10, 64, 1e-8, 1e-10


@pytest.fixture(scope="module")
def state():
    import paper_2406_17823_b300 as P
    (u, v), dx = I.shear_jet(N_BITS, seed=0)
    ctx = P.Context(N_BITS, eps=EPS, chi_max=CHI)
    A = Q.from_dense(u, EPS, CHI)
    B = Q.from_dense(v, EPS, CHI)
    ops = Q.build_operators(N_BITS, dx)
    return ctx, (u, v), A, B, ops


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_from_dense_full_size(state):
    ctx, (u, v), A, B, ops = state
    g = ctx.from_dense(u)
    assert rel(ctx.to_dense(g).cpu().numpy(), Q.to_dense(A)) <= TOL
    assert max(g.bonds) <= CHI


@pytest.mark.parametrize("which", [1, 3])
def test_apply_full_size(state, which):
    ctx, _, A, B, ops = state
    W = ops.D[0] if which == 1 else ops.lap
    g = ctx.apply_mpo(which, ctx.from_cores(A))
    o = Q.apply_mpo(W, A, EPS, CHI)
    assert rel(ctx.to_dense(g).cpu().numpy(), Q.to_dense(o)) <= TOL


def test_hadamard_full_size(state):
    ctx, _, A, B, ops = state
    g = ctx.hadamard(ctx.from_cores(A), ctx.from_cores(B))
    o = Q.hadamard(A, B, EPS, CHI)
    assert rel(ctx.to_dense(g).cpu().numpy(), Q.to_dense(o)) <= TOL


def test_add_full_size(state):
    ctx, _, A, B, ops = state
    g = ctx.add([0.25, -3e-4], [ctx.from_cores(A), ctx.from_cores(B)])
    o = Q.add([0.25, -3e-4], [A, B], EPS, CHI)
    assert rel(ctx.to_dense(g).cpu().numpy(), Q.to_dense(o)) <= TOL


@pytest.fixture(scope="module")
def oracle_two_steps(state):
    """Two oracle RK4 steps of the bench workload (paper solver settings,
    Re = 2e5, dt = 0.1 dx / max|u0|), about a minute of CPU time."""
    _, (u, v), A, B, ops = state
    dx = 2 * np.pi / 2 ** N_BITS
    dt, nu = 0.1 * dx / float(np.abs(u).max()), 1 / 2e5
    o = [A, B]
    prm = Q.Params(eps=EPS, chi_max=CHI)
    for _ in range(2):
        o = Q.rk4_step(o, dt, nu, prm, ops)
    return dt, nu, [Q.to_dense(x) for x in o]


def test_rk4_step_full_size(state, oracle_two_steps):
    """One RK4 step of the bench workload, twice on the GPU so that the
    second step runs from replayed stage graphs, against two oracle steps."""
    import paper_2406_17823_b300 as P
    _, (u, v), A, B, ops = state
    dt, nu, want = oracle_two_steps
    ctx = P.Context(N_BITS, eps=EPS, chi_max=CHI, graphs=1)
    g = [ctx.from_cores(c) for c in (A, B)]
    for _ in range(2):
        ctx.rk4_step(g[0], g[1], dt, nu)
    assert ctx.graph_stats()[1] >= 2
    for got, ref in zip(g, want):
        r = rel(ctx.to_dense(got).cpu().numpy(), ref)
        print(f"full-size RK4, two steps: relative L2 {r:.2e}")
        assert r <= TOL


def test_mixed_rk4_two_steps_full_size(state, oracle_two_steps):
    """The mixed form at the bench configuration, against the oracle itself
    (not through the FP64 GPU path): two RK4 steps with whole-step graphs
    (the bench's mode; the second step replays nothing yet, the graph is
    captured there), within the mixed form's 1e-6 relative L2."""
    import paper_2406_17823_b300 as P
    _, (u, v), A, B, ops = state
    dt, nu, want = oracle_two_steps
    ctx = P.Context(N_BITS, eps=EPS, chi_max=CHI, graphs=2, precision=P.PREC_MIXED)
    g = [ctx.from_cores(c) for c in (A, B)]
    for _ in range(2):
        ctx.rk4_step(g[0], g[1], dt, nu)
    for got, ref in zip(g, want):
        r = rel(ctx.to_dense(got).cpu().numpy(), ref)
        print(f"full-size mixed RK4, two steps: relative L2 {r:.2e}")
        assert r <= 1e-6
