"""Batched trajectories (qtt_rk4_step_batched) against the same steps taken
one trajectory at a time, and one trajectory against the oracle.

Trajectories differ in n, chi_max and initial condition; the batch runs
them concurrently (one host thread and stream set each).  Every kernel is
deterministic, so the batched results must equal the sequential ones bit
for bit.
"""
import numpy as np
import pytest

import qtt_inputs as I
from oracle import qtt as Q

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2406_17823_b300 as P
    return P


CASES = [dict(n=5, chi_max=8, eps=1e-10), dict(n=6, chi_max=16, eps=1e-8),
         dict(n=6, chi_max=32, eps=1e-8)]


def initial(case, i):
    n = case["n"]
    if i == 0:
        return I.taylor_green(n)
    (u, v), dx = I.shear_jet(n, seed=i)
    return [u, v], dx


def test_batched_equals_sequential(P):
    dts, nus, fields = [], [], []
    for i, c in enumerate(CASES):
        f, dx = initial(c, i)
        fields.append(f)
        dts.append(0.1 * dx / float(np.max(np.abs(f[0])) + 1e-30))
        nus.append(1e-3)
    batch = P.Batch(CASES)
    u1 = [batch.contexts[i].from_dense(fields[i][0]) for i in range(len(CASES))]
    u2 = [batch.contexts[i].from_dense(fields[i][1]) for i in range(len(CASES))]
    for _ in range(2):
        assert batch.rk4_step(u1, u2, dts, nus)
    for i, c in enumerate(CASES):
        ctx = P.Context(c["n"], eps=c["eps"], chi_max=c["chi_max"])
        a, b = ctx.from_dense(fields[i][0]), ctx.from_dense(fields[i][1])
        for _ in range(2):
            ctx.rk4_step(a, b, dts[i], nus[i])
        bc = batch.contexts[i]
        for x, y in ((u1[i], a), (u2[i], b)):
            assert np.array_equal(bc.to_dense(x).cpu().numpy(), ctx.to_dense(y).cpu().numpy())


def test_batched_member_matches_oracle(P):
    c = CASES[0]
    f, dx = initial(c, 0)
    dt, nu = 0.01, 0.01
    batch = P.Batch([c, CASES[1]])
    g, dx1 = initial(CASES[1], 1)
    u1 = [batch.contexts[0].from_dense(f[0]), batch.contexts[1].from_dense(g[0])]
    u2 = [batch.contexts[0].from_dense(f[1]), batch.contexts[1].from_dense(g[1])]
    batch.rk4_step(u1, u2, [dt, 0.1 * dx1], [nu, 1e-3])
    prm = Q.Params(eps=c["eps"], chi_max=c["chi_max"])
    ops = Q.build_operators(c["n"], dx)
    u = [Q.from_dense(x, c["eps"], c["chi_max"]) for x in f]
    o = Q.rk4_step(u, dt, nu, prm, ops)
    for got, ref in zip((u1[0], u2[0]), o):
        R = Q.to_dense(ref)
        G = batch.contexts[0].to_dense(got).cpu().numpy()
        assert np.linalg.norm(G - R) <= 1e-10 * np.linalg.norm(R)
