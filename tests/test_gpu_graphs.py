"""Stage right-hand sides replayed as CUDA graphs (params.graphs = 1) against
the same steps launched eagerly.

The graph holds the eager run's kernels with the eager run's arguments and
per-stream order, so every result must equal the eager one bit for bit; the
eager path itself is checked against the oracle elsewhere, and one graph
trajectory is checked against the oracle here as well.
"""
import time

import numpy as np
import pytest

import qtt_inputs as I
from oracle import qtt as Q

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2406_17823_b300 as P
    return P


def dense(ctx, m):
    return ctx.to_dense(m).cpu().numpy()


def run(P, n, chi, eps, steps, graphs, precision=0, scheme="rk4", seed=0):
    (u, v), dx = I.shear_jet(n, seed=seed)
    dt, nu = 0.1 * dx / float(np.abs(u).max()), 1e-4
    ctx = P.Context(n, eps=eps, chi_max=chi, precision=precision, graphs=graphs)
    a, b = ctx.from_dense(u), ctx.from_dense(v)
    step = ctx.rk4_step if scheme == "rk4" else ctx.euler_step
    counts = []
    for _ in range(steps):
        before = ctx.stats()["launches"]
        step(a, b, dt, nu)
        ctx.sync()
        counts.append(ctx.stats()["launches"] - before)
    return ctx, a, b, counts


@pytest.mark.parametrize("precision", [0, 1])
def test_graph_steps_equal_eager(P, precision):
    """Four RK4 steps.  Stages 1 and 2 share a key (same h and capacities):
    a key is captured at its second occurrence and replayed from its third,
    so once the capacities have settled (after the first step) every stage
    of step 4 is a replay."""
    c0, a0, b0, n0 = run(P, 7, 32, 1e-8, 4, graphs=0, precision=precision)
    c1, a1, b1, n1 = run(P, 7, 32, 1e-8, 4, graphs=1, precision=precision)
    for x, y in ((a0, a1), (b0, b1)):
        assert np.array_equal(dense(c0, x), dense(c1, y))
    captured, replays = c1.graph_stats()
    assert captured >= 3 and replays >= 4
    assert c0.graph_stats() == (0, 0)
    # a replayed stage counts the kernels its graph holds
    assert n1[-1] == n0[-1]


def test_graph_euler_equal_eager(P):
    c0, a0, b0, _ = run(P, 6, 16, 1e-8, 4, graphs=0, scheme="euler", seed=3)
    c1, a1, b1, _ = run(P, 6, 16, 1e-8, 4, graphs=1, scheme="euler", seed=3)
    for x, y in ((a0, a1), (b0, b1)):
        assert np.array_equal(dense(c0, x), dense(c1, y))
    assert c1.graph_stats()[1] >= 1


def test_graph_trajectory_matches_oracle(P):
    n, chi, eps = 5, 16, 1e-10
    (u, v), dx = I.shear_jet(n, seed=1)
    dt, nu = 0.1 * dx / float(np.abs(u).max()), 1e-3
    ctx = P.Context(n, eps=eps, chi_max=chi, graphs=1)
    a, b = ctx.from_dense(u), ctx.from_dense(v)
    prm = Q.Params(eps=eps, chi_max=chi)
    ops = Q.build_operators(n, dx)
    o = [Q.from_dense(f, eps, chi) for f in (u, v)]
    for _ in range(3):
        ctx.rk4_step(a, b, dt, nu)
        o = Q.rk4_step(o, dt, nu, prm, ops)
    assert ctx.graph_stats()[1] >= 2
    for got, ref in zip((a, b), o):
        R = Q.to_dense(ref)
        assert np.linalg.norm(dense(ctx, got) - R) <= 1e-10 * np.linalg.norm(R)


def test_graphs_follow_parameter_changes(P):
    """set_params drops the captured graphs: a changed eps takes effect."""
    n = 6
    (u, v), dx = I.shear_jet(n, seed=2)
    dt, nu = 0.1 * dx / float(np.abs(u).max()), 1e-4
    g = P.Context(n, eps=1e-8, chi_max=16, graphs=1)
    e = P.Context(n, eps=1e-8, chi_max=16)
    ga, gb = g.from_dense(u), g.from_dense(v)
    ea, eb = e.from_dense(u), e.from_dense(v)
    for ctx, a, b in ((g, ga, gb), (e, ea, eb)):
        for _ in range(2):
            ctx.rk4_step(a, b, dt, nu)
        ctx.set_params(eps=1e-4, chi_max=8)
        for _ in range(2):
            ctx.rk4_step(a, b, dt, nu)
    for x, y in ((ga, ea), (gb, eb)):
        assert np.array_equal(dense(g, x), dense(e, y))
    assert max(ga.bonds) <= 8
    assert g.graph_stats()[0] >= 1


@pytest.mark.parametrize("graphs", [1, 2])
def test_batched_graphs_equal_sequential(P, graphs):
    cases = [dict(n=5, chi_max=8, eps=1e-10, graphs=graphs),
             dict(n=6, chi_max=16, eps=1e-8, graphs=graphs)]
    fields, dts = [], []
    for i, c in enumerate(cases):
        (u, v), dx = I.shear_jet(c["n"], seed=10 + i)
        fields.append((u, v))
        dts.append(0.1 * dx / float(np.abs(u).max()))
    nus = [1e-3, 1e-3]
    batch = P.Batch(cases)
    u1 = [batch.contexts[i].from_dense(fields[i][0]) for i in range(2)]
    u2 = [batch.contexts[i].from_dense(fields[i][1]) for i in range(2)]
    for _ in range(4):
        assert batch.rk4_step(u1, u2, dts, nus)
    assert all(c.graph_stats()[1] >= 4 for c in batch.contexts)
    for i, c in enumerate(cases):
        ctx = P.Context(c["n"], eps=c["eps"], chi_max=c["chi_max"])
        a, b = ctx.from_dense(fields[i][0]), ctx.from_dense(fields[i][1])
        for _ in range(4):
            ctx.rk4_step(a, b, dts[i], nus[i])
        bc = batch.contexts[i]
        for x, y in ((u1[i], a), (u2[i], b)):
            assert np.array_equal(bc.to_dense(x).cpu().numpy(), dense(ctx, y))


def test_graph_timing_small_grid(P):
    """Host-bound case (Taylor-Green, 2^6 x 2^6, chi 16): steps per second
    eager, with stage graphs and with step graphs (printed; timings on a
    shared GPU are not asserted)."""
    import torch
    res = {}
    for graphs in (0, 1, 2):
        (u, v), dx = I.taylor_green(6)
        ctx = P.Context(6, eps=1e-12, chi_max=16, graphs=graphs)
        a, b = ctx.from_dense(u), ctx.from_dense(v)
        for _ in range(3):
            ctx.rk4_step(a, b, 1e-3, 0.01)
        ctx.sync()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(10):
            ctx.rk4_step(a, b, 1e-3, 0.01)
        ctx.sync()
        res[graphs] = 10 / (time.perf_counter() - t0)
    print(f"Taylor-Green 2^6, chi 16: eager {res[0]:.1f} steps/s, stage graphs {res[1]:.1f}, "
          f"step graphs {res[2]:.1f}")
    assert all(r > 0 for r in res.values())


def test_upload_keeps_capacities_and_replays(P):
    """A state read back to host memory and uploaded into the same objects
    keeps its capacities: the next step replays every stage and equals the
    eager context doing the same."""
    out = []
    for graphs in (0, 1):
        (u, v), dx = I.shear_jet(6, seed=4)
        dt, nu = 0.1 * dx / float(np.abs(u).max()), 1e-4
        ctx = P.Context(6, eps=1e-8, chi_max=16, graphs=graphs)
        a, b = ctx.from_dense(u), ctx.from_dense(v)
        for _ in range(4):
            ctx.rk4_step(a, b, dt, nu)
        host = [ctx.to_cores(a), ctx.to_cores(b)]
        before = ctx.graph_stats()[1]
        for m, c in zip((a, b), host):
            ctx.upload_cores(m, c)
        ctx.rk4_step(a, b, dt, nu)
        if graphs:
            assert ctx.graph_stats()[1] - before == 4
        out.append((dense(ctx, a), dense(ctx, b)))
    for x, y in zip(*out):
        assert np.array_equal(x, y)


def test_upload_rejects_bond_above_capacity(P):
    """Capacities never exceed chi_max: a bond of chi_max + 1 is refused."""
    ctx = P.Context(5, eps=1e-8, chi_max=4)
    (u, v), dx = I.shear_jet(5, seed=0)
    a = ctx.from_dense(u)
    bonds = [1, 4, 5, 4, 4, 1]
    wide = [np.zeros((bonds[k], 4, bonds[k + 1])) for k in range(5)]
    with pytest.raises(P.QttError):
        ctx.upload_cores(a, wide)


@pytest.mark.parametrize("precision", [0, 1])
def test_step_graph_equals_eager(P, precision):
    """graphs = 2: the whole RK4 step (stages, projection with its CG and
    sweep loops as device-driven WHILE nodes, final sum) is one replayed
    graph from the third step on; fields, converged flags and CG iteration
    counts equal the eager run's."""
    res = []
    for graphs in (0, 2):
        (u, v), dx = I.shear_jet(7, seed=5)
        dt, nu = 0.1 * dx / float(np.abs(u).max()), 1e-4
        ctx = P.Context(7, eps=1e-8, chi_max=32, precision=precision, graphs=graphs)
        a, b = ctx.from_dense(u), ctx.from_dense(v)
        conv, cg, nl = [], [], []
        for _ in range(4):
            before = ctx.stats()
            conv.append(ctx.rk4_step(a, b, dt, nu))
            after = ctx.stats()
            cg.append(after["cg_iters"] - before["cg_iters"])
            nl.append(after["launches"] - before["launches"])
        res.append((dense(ctx, a), dense(ctx, b), conv, cg, nl, ctx.graph_stats()))
    (a0, b0, c0, g0, l0, _), (a1, b1, c1, g1, l1, gs) = res
    assert gs[1] >= 2  # steps 3 and 4 replayed
    assert np.array_equal(a0, a1) and np.array_equal(b0, b1)
    assert c0 == c1 and g0 == g1
    # kernels run by a replayed step (loop bodies counted per pass on the
    # device): the eager step's count less the no-op CG iterations its
    # host loop launches past convergence, plus one condition per pass
    print(f"kernels per step: eager {l0[-1]}, step graph {l1[-1]}")
    assert 0.5 * l0[-1] < l1[-1] < 1.5 * l0[-1]


def test_step_graph_reports_caps(P):
    """A CG cap of one iteration: every replayed step reports that a
    projection reached its cap, as the eager step does."""
    (u, v), dx = I.shear_jet(6, seed=6)
    dt, nu = 0.1 * dx / float(np.abs(u).max()), 1e-4
    out = []
    for graphs in (0, 2):
        ctx = P.Context(6, eps=1e-8, chi_max=16, cg_tol=1e-14, cg_maxit=1, graphs=graphs)
        a, b = ctx.from_dense(u), ctx.from_dense(v)
        out.append([ctx.rk4_step(a, b, dt, nu) for _ in range(4)])
        if graphs:
            assert ctx.graph_stats()[1] >= 2
    assert out[0] == out[1] == [False] * 4


def test_step_graph_timing(P):
    """2^7 jet, chi 32: steps per second with stage graphs and with whole-step
    graphs (printed)."""
    import torch
    res = {}
    for graphs in (1, 2):
        (u, v), dx = I.shear_jet(7, seed=7)
        dt, nu = 0.1 * dx / float(np.abs(u).max()), 1e-4
        ctx = P.Context(7, eps=1e-8, chi_max=32, graphs=graphs)
        a, b = ctx.from_dense(u), ctx.from_dense(v)
        for _ in range(3):
            ctx.rk4_step(a, b, dt, nu)
        ctx.sync()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(5):
            ctx.rk4_step(a, b, dt, nu)
        ctx.sync()
        res[graphs] = 5 / (time.perf_counter() - t0)
    print(f"2^7 jet, chi 32: stage graphs {res[1]:.2f} steps/s, step graphs {res[2]:.2f} steps/s")
