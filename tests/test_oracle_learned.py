"""Pins of the learned-truncation oracle (CPU only).

The generator against its published output stream and its moments; the
range finder against the exact residual |M - Q Q^T M|_F, against the plain
compression when it spans M, and its fallback rule; the perceptron's
back-propagation against central differences; Adam's first step against
its closed form.
"""
import os

import numpy as np
import pytest

import qtt_inputs as I
from oracle import learned as Lr
from oracle import qtt as Q

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_published_stream():
    vals = [int(l) for l in open(os.path.join(GOLD, "splitmix64_seed1234567.txt"))
            if l.strip() and not l.startswith("#")]
    assert [Lr.bits(1234567, i) for i in range(len(vals))] == vals


def test_gaussian_moments():
    g = np.array([Lr.gaussian(Lr.bond_key(3, 1, 2), e) for e in range(20000)])
    assert abs(g.mean()) < 0.03
    assert abs(g.var() - 1.0) < 0.04
    assert abs(np.mean(g ** 3)) < 0.1          # symmetric
    assert abs(np.mean(g ** 4) - 3.0) < 0.2    # Gaussian kurtosis


def test_trunc_rank_total_reduces_to_plain_rule():
    rng = np.random.default_rng(1)
    for _ in range(20):
        s = np.sort(np.abs(rng.standard_normal(12)) * np.logspace(0, -9, 12))[::-1]
        for eps in (1e-2, 1e-5, 1e-8):
            assert Lr.trunc_rank_total(s, 0.0, eps, 8) == Q.trunc_rank(s, eps, 8)


def test_range_finder_estimate_is_exact_residual():
    rng = np.random.default_rng(2)
    M = rng.standard_normal((40, 9)) @ rng.standard_normal((9, 64))
    M += 1e-3 * rng.standard_normal((40, 64))
    for w in (4, 9, 20):
        Qm, B, outside = Lr.range_finder(M, w, Lr.bond_key(0, 0, 5))
        res = M - Qm @ (Qm.T @ M)
        exact = float(np.sum(res * res))
        assert abs(outside - exact) <= 1e-12 * float(np.sum(M * M))
        assert np.allclose(Qm.T @ Qm, np.eye(Qm.shape[1]), atol=1e-13)


def test_range_finder_equals_full_svd_when_it_spans_the_state():
    n = 6
    A = Q.from_dense(I.random_field(n, seed=7), 1e-12, 64)   # smooth: small ranks
    ranks = Q.bond_dims(A)
    widths = {b: ranks[b] + 4 for b in range(1, n)}
    info = []
    # eps^2 well above the rounding floor of |M|^2 - |B|^2 (about 1e-16 |M|^2)
    R = Lr.compress_rf(A, 1e-6, 64, widths, seed=1, info=info)
    P = Q.compress(A, 1e-6, 64)
    assert all(u for (_, u, _, _) in info)
    assert np.linalg.norm(Q.to_dense(R) - Q.to_dense(P)) <= 1e-12 * np.linalg.norm(Q.to_dense(P))


def test_fallback_when_the_sketch_misses_weight():
    n = 6
    A = Q.from_dense(I.white_field(n, seed=3), 0.0, 64)       # full-rank noise
    widths = {b: 2 for b in range(1, n)}
    info = []
    R = Lr.compress_rf(A, 1e-8, 64, widths, seed=0, info=info)
    P = Q.compress(A, 1e-8, 64)
    eps = 1e-8
    for (_, used, outside, nM) in info:
        assert used == (not outside > Lr.ACCEPT * eps * eps * nM)
    assert any(not u for (_, u, _, _) in info)
    # every bond here needs more than two directions: all fell back
    assert np.linalg.norm(Q.to_dense(R) - Q.to_dense(P)) <= 1e-12 * np.linalg.norm(Q.to_dense(P))


def test_mlp_gradient_central_differences():
    rng = np.random.default_rng(4)
    p = Lr.init_params(5) + 0.01 * rng.standard_normal(Lr.N_PARAM)
    X = rng.uniform(-1, 0, (17, Lr.N_FEAT))
    y = rng.uniform(0, 1, 17)
    L, g = Lr.loss_and_grad(p, X, y)
    assert abs(L - float(np.mean((Lr.forward(p, X) - y) ** 2))) < 1e-14
    h = 1e-6
    idx = rng.choice(Lr.N_PARAM, 40, replace=False).tolist() + [Lr.N_PARAM - 1]
    for i in idx:
        e = np.zeros(Lr.N_PARAM)
        e[i] = h
        fd = (Lr.loss_and_grad(p + e, X, y)[0] - Lr.loss_and_grad(p - e, X, y)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i]))


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(6)
    p = rng.standard_normal(10)
    g = rng.standard_normal(10)
    p1, m, v = Lr.adam_step(p, g, np.zeros(10), np.zeros(10), 1, 1e-3)
    # bias-corrected first moments equal g, second |g|^2: a step of lr * sign(g)
    assert np.allclose(p1, p - 1e-3 * g / (np.abs(g) + 1e-8), atol=1e-15)


def test_features_layout():
    s = np.array([4.0, 2.0, 0.4, 0.0])
    f = Lr.features(s, 3, 10)
    assert f.shape == (33,)
    assert f[0] == 0.0
    assert abs(f[1] - np.log10(0.5) / 16) < 1e-15
    assert f[3] == -1.0 and f[31] == -1.0      # zero and missing values clip at -16
    assert f[32] == pytest.approx(0.3)
