"""Learned truncation on the GPU against the oracle (oracle/learned.py).

* the range finder's Gaussian test matrix, entry by entry;
* the perceptron's forward pass, loss and gradient (FP32 kernels against the
  FP64 oracle) and Adam steps;
* the range-finder compression with a given predicted rank against the
  oracle's compress_rf (same test matrix, same fallback rule), and against
  the plain compression at the learned form's 1e-6 bar;
* a trained predictor on a turbulence trajectory: how many cuts it serves
  without the full SVD, its error against the plain FP64 form, and its time.
"""
import time

import numpy as np
import pytest

import qtt_inputs as I
from oracle import learned as Lr
from oracle import qtt as Q

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2406_17823_b300 as P
    return P


@pytest.fixture(scope="module")
def torch():
    import torch
    return torch


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_rf_omega_matches_oracle(P):
    ctx = P.Context(4)
    for key, D, w in [(Lr.bond_key(0, 0, 3), 5, 7), (Lr.bond_key(0, 17, 9), 3, 20)]:
        g = ctx.rf_omega(key, D, w).cpu().numpy()
        o = Lr.omega(key, 4 * D, w)
        assert np.max(np.abs(g - o)) <= 1e-13 * max(1.0, np.max(np.abs(o)))


def test_mlp_forward_loss_grad_vs_oracle(P, torch):
    rng = np.random.default_rng(0)
    p = Lr.init_params(1) + 0.05 * rng.standard_normal(Lr.N_PARAM)
    X = rng.uniform(-1, 0, (257, Lr.N_FEAT))
    y = rng.uniform(0, 1, 257)
    ctx = P.Context(4)
    pt = torch.tensor(p, dtype=torch.float32, device="cuda")
    Xt = torch.tensor(X, dtype=torch.float32, device="cuda")
    yt = torch.tensor(y, dtype=torch.float32, device="cuda")
    out = ctx.mlp_forward(pt, Xt).cpu().numpy()
    p32 = pt.cpu().numpy().astype(np.float64)
    X32 = Xt.cpu().numpy().astype(np.float64)
    y32 = yt.cpu().numpy().astype(np.float64)
    ref = Lr.forward(p32, X32)
    assert np.max(np.abs(out - ref)) <= 1e-5 * max(1.0, np.max(np.abs(ref)))
    L, g = ctx.mlp_loss_grad(pt, Xt, yt)
    Lo, go = Lr.loss_and_grad(p32, X32, y32)
    assert abs(float(L.cpu()) - Lo) <= 1e-5 * Lo
    g = g.cpu().numpy()
    assert np.linalg.norm(g - go) <= 1e-5 * np.linalg.norm(go)


def test_mlp_adam_steps_vs_oracle(P, torch):
    rng = np.random.default_rng(2)
    p = Lr.init_params(3)
    X = rng.uniform(-1, 0, (64, Lr.N_FEAT))
    y = 0.3 + 0.2 * X[:, 0]
    ctx = P.Context(4)
    pt = torch.tensor(p, dtype=torch.float32, device="cuda")
    Xt = torch.tensor(X, dtype=torch.float32, device="cuda")
    yt = torch.tensor(y, dtype=torch.float32, device="cuda")
    p64 = pt.cpu().numpy().astype(np.float64)
    X64 = Xt.cpu().numpy().astype(np.float64)
    y64 = yt.cpu().numpy().astype(np.float64)
    losses = ctx.mlp_train(pt, Xt, yt, 5, 1e-3).cpu().numpy()
    m = np.zeros_like(p64)
    v = np.zeros_like(p64)
    for t in range(1, 6):
        Lo, g = Lr.loss_and_grad(p64, X64, y64)
        assert abs(losses[t - 1] - Lo) <= 1e-4 * Lo
        p64, m, v = Lr.adam_step(p64, g, m, v, t, 1e-3)
    assert np.max(np.abs(pt.cpu().numpy() - p64)) <= 2e-6


def constant_predictor(rank, chi):
    """Parameters whose output is rank / chi for every input (exact in FP32
    for the ranks used here), so the predicted rank is known exactly."""
    p = np.zeros(Lr.N_PARAM)
    p[-1] = rank / chi
    return p


@pytest.mark.parametrize("rank", [6, 20])
def test_range_finder_compress_vs_oracle(P, torch, rank):
    n, chi, eps = 7, 32, 1e-6
    u, _ = I.decaying_turbulence(n, 4, seed=1)
    A = Q.from_dense(u[0] + 1e-3 * I.white_field(n, seed=2), 0.0, 64)
    ctx = P.Context(n, eps=eps, chi_max=chi, learned_trunc=P.LEARNED_ON, rf_oversample=6,
                    rf_min_width=1)
    pc = constant_predictor(rank, chi)
    ctx.learned_set(torch.tensor(pc, dtype=torch.float32, device="cuda"))
    # first call: no features yet -> every cut is the full SVD (slot 0)
    ctx.learned_next_step()
    g0 = ctx.compress(ctx.from_cores(A), eps, chi)
    ref = Q.to_dense(Q.compress(A, eps, chi))
    assert rel(ctx.to_dense(g0).cpu().numpy(), ref) <= 1e-10
    acc0, fb0 = ctx.learned_stats()
    # second call in slot 0 of the next step: range finder of width rank + 6
    ctx.learned_next_step()
    g1 = ctx.compress(ctx.from_cores(A), eps, chi)
    acc1, fb1 = ctx.learned_stats()
    widths = {b: min(rank, chi) + 6 for b in range(1, n)}
    info = []
    o = Lr.compress_rf(A, eps, chi, widths, seed=0, slot=0, info=info)
    d1 = ctx.to_dense(g1).cpu().numpy()
    assert rel(d1, Q.to_dense(o)) <= 1e-10
    n_rf = sum(1 for t in info if t[1])
    assert acc1 - acc0 == n_rf and fb1 - fb0 == len(info) - n_rf
    # the learned form's bar against the plain compression
    assert rel(d1, ref) <= 1e-6
    print(f"rank {rank}: {n_rf} of {len(info)} cuts by the range finder")


def collect(ctx, nsteps, u, dt, nu):
    """Run nsteps in LOG mode; return training pairs (features of step t,
    rank / chi of step t + 1) over every (slot, bond) cut in both steps."""
    X, Y = [], []
    prev = None
    for _ in range(nsteps):
        ctx.rk4_step(u[0], u[1], dt, nu)
        f, r, ns = ctx.learned_log()
        if prev is not None:
            pf, pr, pns = prev
            m = min(ns, pns)
            ok = (pr[:m] > 0) & (r[:m] > 0)
            X.append(pf[:m][ok])
            Y.append(r[:m][ok] / ctx.params.chi_max)
        prev = (f, r, ns)
    return np.concatenate(X), np.concatenate(Y)


def test_trained_predictor_gain(P, torch):
    n, chi, eps = 7, 32, 1e-6
    u0, dx = I.decaying_turbulence(n, 4, seed=3)
    dt = 0.2 * dx / float(np.max(np.abs(u0)))
    nu = 1e-4
    # training data from the plain method's own cuts
    log = P.Context(n, eps=eps, chi_max=chi, learned_trunc=P.LEARNED_LOG)
    st = [log.from_dense(f) for f in u0]
    X, Y = collect(log, 4, st, dt, nu)
    assert X.shape[0] > 100
    pt = torch.tensor(Lr.init_params(0), dtype=torch.float32, device="cuda")
    Xt = torch.tensor(X, dtype=torch.float32, device="cuda")
    Yt = torch.tensor(Y, dtype=torch.float32, device="cuda")
    p_untrained = pt.clone()
    losses = log.mlp_train(pt, Xt, Yt, 800, 3e-3).cpu().numpy()
    assert losses[-1] < 0.2 * losses[0]
    # continue the trajectory three ways from the same state: plain cuts,
    # the trained predictor, and the untrained one (what training gains)
    cores = [log.to_cores(m) for m in st]

    def run(ctx):
        m = [ctx.from_cores(c) for c in cores]
        ctx.rk4_step(m[0], m[1], dt, nu)   # fills the features of every slot
        a0 = ctx.learned_stats() if ctx.params.learned_trunc else (0, 0)
        ctx.sync()
        t0 = time.perf_counter()
        for _ in range(2):
            ctx.rk4_step(m[0], m[1], dt, nu)
        ctx.sync()
        t = time.perf_counter() - t0
        a1 = ctx.learned_stats() if ctx.params.learned_trunc else (0, 0)
        acc, fb = a1[0] - a0[0], a1[1] - a0[1]
        return m, t, acc / max(1, acc + fb)

    plain = P.Context(n, eps=eps, chi_max=chi)
    a, t_plain, _ = run(plain)
    res = {}
    for name, prm in (("trained", pt), ("untrained", p_untrained)):
        ctx = P.Context(n, eps=eps, chi_max=chi, learned_trunc=P.LEARNED_ON, rf_oversample=8,
                        rf_min_width=1)
        ctx.learned_set(prm)
        b, t, served = run(ctx)
        err = max(rel(ctx.to_dense(b[i]).cpu().numpy(), plain.to_dense(a[i]).cpu().numpy())
                  for i in range(2))
        res[name] = (served, err, t)
        print(f"{name}: range finder served {served:.2f} of the cuts; error vs plain "
              f"{err:.2e}; 2 steps {t:.3f} s (plain {t_plain:.3f} s)")
    print(f"training loss {losses[0]:.3e} -> {losses[-1]:.3e}")
    assert res["trained"][0] >= 0.5
    assert res["trained"][0] > res["untrained"][0]
    assert res["trained"][1] <= 1e-6 and res["untrained"][1] <= 1e-6
