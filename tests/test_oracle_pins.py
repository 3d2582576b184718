"""Pins of the CPU oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: the
paper's printed carry table, brute-force dense stencils, closed forms,
Eckart-Young, exact Fourier-space solves and exact invariants.
"""
import math
import os

import numpy as np
import pytest

import qtt_inputs as I
from oracle import dense as Dn
from oracle import qtt as Q

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
FULL = 10 ** 9
TIGHT = dict(cg_tol=1e-13, cg_maxit=2000, sweep_tol=1e-14, max_sweeps=40)


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


# ---------------------------------------------------------------- App. A
def test_carry_table_matches_paper():
    """App. A, Table "diff_mpo": the 12 non-zero entries, value 1."""
    rows = [list(map(int, l.split())) for l in open(os.path.join(GOLDEN, "diff_mpo_table.txt"))
            if l.strip() and not l.startswith("#")]
    C = Q.carry_core(1)
    want = np.zeros_like(C)
    for am, am1, w, wp, val in rows:
        want[am, w, wp, am1] = val
    assert len(rows) == 12
    np.testing.assert_array_equal(C, want)


@pytest.mark.parametrize("n", [3, 4, 5])
@pytest.mark.parametrize("axis", [1, 2])
def test_diff_mpo_equals_stencil_bruteforce(n, axis):
    """Eq. "fdm2": dense matrix of the MPO == periodic central stencil."""
    N = 2 ** n
    dx = 2 * math.pi / N
    M = Q.mpo_to_dense(Q.mpo_diff(n, axis, dx))
    S = np.zeros((N * N, N * N))
    for x1 in range(N):
        for x2 in range(N):
            r = x1 * N + x2
            if axis == 1:
                S[r, ((x1 + 1) % N) * N + x2] += 1 / (2 * dx)
                S[r, ((x1 - 1) % N) * N + x2] -= 1 / (2 * dx)
            else:
                S[r, x1 * N + (x2 + 1) % N] += 1 / (2 * dx)
                S[r, x1 * N + (x2 - 1) % N] -= 1 / (2 * dx)
    assert np.abs(M - S).max() <= 1e-13 / dx
    # App. B uses D^T = -D
    assert np.abs(M + M.T).max() == 0.0


def test_second_order_operators_bruteforce():
    """Laplacian D1 D1 + D2 D2 (App. B, Eq. for B_i) and the projection
    blocks D_i^T D_j (Eq. big_LS) against stencil compositions."""
    n = 4
    N = 2 ** n
    dx = 2 * math.pi / N
    ops = Q.build_operators(n, dx)
    F = I.white_field(n, seed=5)
    f = F.reshape(-1)
    lap = sum(Dn.d(Dn.d(F, j, dx), j, dx) for j in (1, 2))
    assert rel(Q.mpo_to_dense(ops.lap) @ f, lap.reshape(-1)) < 1e-13
    for i in range(2):
        for j in range(2):
            want = -Dn.d(Dn.d(F, j + 1, dx), i + 1, dx)
            assert rel(Q.mpo_to_dense(ops.K[(i, j)]) @ f, want.reshape(-1)) < 1e-13
    assert max(w.shape[3] for w in ops.lap) <= 5
    assert max(w.shape[3] for w in ops.K[(0, 0)]) <= 3


def test_derivative_of_sine_closed_form():
    """D1 sin(k x) = (sin(k dx)/dx) cos(k x), exactly, through the QTT."""
    n = 7
    X1, X2, dx = I.grid(n)
    ops = Q.build_operators(n, dx)
    for k in (1, 3):
        q = Q.from_dense(np.sin(k * X1) * np.cos(X2), 1e-14, 64)
        out = Q.to_dense(Q.apply_mpo(ops.D[0], q, 0.0, FULL))
        want = math.sin(k * dx) / dx * np.cos(k * X1) * np.cos(X2)
        assert rel(out, want) < 1e-13
        out2 = Q.to_dense(Q.apply_mpo(ops.lap, q, 0.0, FULL))
        c1, c2 = (math.sin(k * dx) / dx) ** 2, (math.sin(dx) / dx) ** 2
        assert rel(out2, -(c1 + c2) * np.sin(k * X1) * np.cos(X2)) < 1e-12


# ------------------------------------------------------------- encoding
def _numerical_ranks(F, tol=1e-12):
    """Schmidt ranks of a dense field at every bond, by plain SVD of the
    reshaped omega tensor (independent of the TT-SVD sweep)."""
    n = int(round(math.log2(F.shape[0])))
    T = Q.dense_to_tensor(F).reshape(-1)
    ranks = []
    for k in range(1, n):
        s = np.linalg.svd(T.reshape(4 ** k, -1), compute_uv=False)
        ranks.append(int(np.sum(s > tol * s[0])))
    return ranks


def test_low_rank_sines_and_cosines():
    """Separable single-axis sines / cosines have QTT rank 2 (Sec. III.F:
    fields with few Fourier modes are low-rank); Taylor-Green
    sin x cos y has rank <= 4."""
    n = 7
    X1, X2, _ = I.grid(n)
    for F in (np.sin(3 * X1), np.cos(2 * X2), np.sin(X1 + X2), np.cos(5 * X1 - 2 * X2)):
        q = Q.from_dense(F, 1e-13, 64)
        assert max(Q.bond_dims(q)) == 2
        assert Q.bond_dims(q)[1:-1] == _numerical_ranks(F)
        assert rel(Q.to_dense(q), F) < 1e-13
    tg = np.sin(X1) * np.cos(X2)
    q = Q.from_dense(tg, 1e-13, 64)
    assert max(Q.bond_dims(q)) <= 4
    assert rel(Q.to_dense(q), tg) < 1e-13


def test_tt_svd_error_bound_and_roundtrip():
    """Each bond discards at most eps^2 of its weight, so the total error is
    at most sqrt(n-1) eps (Sec. III.E); eps = 0 is a lossless round trip."""
    n = 6
    F = I.white_field(n, seed=1) * 0.01 + I.random_field(n, seed=2)
    assert rel(Q.to_dense(Q.from_dense(F, 0.0, FULL)), F) < 1e-14
    for eps in (1e-2, 1e-4):
        q = Q.from_dense(F, eps, FULL)
        assert rel(Q.to_dense(q), F) <= math.sqrt(n - 1) * eps
    assert Q.bond_dims(Q.from_dense(F, 0.0, 7))[3] == 7


def test_trunc_rank_rule():
    s = np.array([1.0, 1e-3, 1e-6, 0.0])
    assert Q.trunc_rank(s, 0.0, 10) == 3            # zeros dropped, nothing else
    assert Q.trunc_rank(s, 1e-5, 10) == 2           # 1e-12 <= 1e-10
    assert Q.trunc_rank(s, 2e-3, 10) == 1
    assert Q.trunc_rank(s, 0.0, 2) == 2             # chi cap
    assert Q.trunc_rank(np.zeros(3), 0.1, 5) == 1


def test_compress_single_cut_is_eckart_young():
    """A compression that truncates one bond only leaves exactly the
    discarded Schmidt weight (Eckart-Young), computed here by a dense SVD."""
    n = 4
    A = I.random_cores(n, [1, 4, 16, 4, 1], seed=3)
    F = Q.to_dense(A)
    T = Q.dense_to_tensor(F).reshape(16, 16)
    s = np.linalg.svd(T, compute_uv=False)
    out = Q.to_dense(Q.compress(A, 0.0, 9))
    assert abs(np.linalg.norm(out - F) - math.sqrt(np.sum(s[9:] ** 2))) < 1e-12 * np.linalg.norm(F)
    assert np.linalg.norm(out) <= np.linalg.norm(F) * (1 + 1e-14)


# ------------------------------------------------------------- MPS algebra
@pytest.mark.parametrize("n", [5, 6])
def test_exact_ops_match_dense(n):
    """With eps = 0 and no cap, apply / add / Hadamard equal their dense
    definitions (stencil, linear combination, element-wise product)."""
    X1, X2, dx = I.grid(n)
    ops = Q.build_operators(n, dx)
    F = I.random_field(n, seed=10)
    G = I.random_field(n, seed=11) + 0.1 * np.sin(7 * X1) * np.cos(3 * X2)
    a = Q.from_dense(F, 0.0, FULL)
    b = Q.from_dense(G, 0.0, FULL)
    assert rel(Q.to_dense(Q.apply_mpo(ops.D[1], a, 0.0, FULL)), Dn.d(F, 2, dx)) < 1e-12
    assert rel(Q.to_dense(Q.add([0.3, -2.0], [a, b], 0.0, FULL)), 0.3 * F - 2.0 * G) < 1e-13
    assert rel(Q.to_dense(Q.hadamard(a, b, 0.0, FULL)), F * G) < 1e-12
    assert rel(Q.to_dense(Q.hadamard_exact(a, b)), F * G) < 1e-13


def test_hadamard_truncation_reaches_rank_product():
    """The zip-up with cap chi keeps everything when rank(a)*rank(b) <= chi."""
    n = 7
    X1, X2, _ = I.grid(n)
    F, G = np.sin(X1) * np.cos(2 * X2), np.cos(3 * X1) + np.sin(X2)
    a, b = Q.from_dense(F, 1e-13, 64), Q.from_dense(G, 1e-13, 64)
    out = Q.hadamard(a, b, 1e-12, 16)
    assert rel(Q.to_dense(out), F * G) < 1e-12


def test_convection_is_energy_neutral():
    """sum_i <u_i, conv_i(u)> = 0 for any u, since D^T = -D (App. B,
    skew-symmetric convection): pins the signs of the Hadamard / MPO
    composition."""
    n = 5
    X1, X2, dx = I.grid(n)
    ops = Q.build_operators(n, dx)
    u = [I.random_field(n, seed=20), I.random_field(n, seed=21)]
    uq = [Q.from_dense(f, 0.0, FULL) for f in u]
    total, scale = 0.0, 0.0
    for i in range(2):
        conv = None
        for j in range(2):
            t1 = Q.hadamard(uq[j], Q.apply_mpo(ops.D[j], uq[i], 0.0, FULL), 0.0, FULL)
            t2 = Q.apply_mpo(ops.D[j], Q.hadamard(uq[j], uq[i], 0.0, FULL), 0.0, FULL)
            part = Q.add([0.5, 0.5], [t1, t2], 0.0, FULL)
            conv = part if conv is None else Q.add([1.0, 1.0], [conv, part], 0.0, FULL)
        total += Q.inner(uq[i], conv)
        scale += math.sqrt(Q.norm2(uq[i]) * Q.norm2(conv))
        assert rel(Q.to_dense(conv), Dn.convection(u, dx)[i]) < 1e-12
    assert abs(total) < 1e-13 * scale


# ------------------------------------------------------------- projection
@pytest.mark.parametrize("h", [1e-3, 1e-2])
def test_projection_equals_fourier_solve(h):
    """At full rank the sweep reaches the exact minimiser of Theta, i.e.
    (I + mu h^2 G^T G)^{-1} w solved per Fourier mode (Eq. big_LS)."""
    n = 4
    X1, X2, dx = I.grid(n)
    ops = Q.build_operators(n, dx)
    w = [I.white_field(n, seed=30), I.white_field(n, seed=31)]
    wq = [Q.from_dense(f, 0.0, FULL) for f in w]
    p = Q.Params(eps=0.0, chi_max=FULL, **TIGHT)
    v, info = Q.project(wq, h, p, ops)
    vd = Dn.project(w, h, p.mu, dx)
    assert info.converged
    for i in range(2):
        assert rel(Q.to_dense(v[i]), vd[i]) < 1e-10


def test_projection_invariants_dense():
    """The exact projection is a contraction and damps the divergence of
    each Fourier mode by exactly 1 / (1 + mu h^2 |g(k)|^2)."""
    n = 5
    _, _, dx = I.grid(n)
    w = [I.white_field(n, seed=40), I.white_field(n, seed=41)]
    h, mu = 1e-3, 2.5e5
    v = Dn.project(w, h, mu, dx)
    assert sum(np.sum(x ** 2) for x in v) <= sum(np.sum(x ** 2) for x in w)
    g1, g2 = Dn.symbols(2 ** n, dx)
    dv, dw = np.fft.fft2(Dn.divergence(v, dx)), np.fft.fft2(Dn.divergence(w, dx))
    np.testing.assert_allclose(dv, dw / (1 + mu * h * h * (abs(g1) ** 2 + abs(g2) ** 2)),
                               atol=1e-9 * np.abs(dw).max())
    vl = Dn.project(w, h, 1e14, dx)
    assert np.abs(Dn.divergence(vl, dx)).max() < 1e-6 * np.abs(Dn.divergence(w, dx)).max()


def test_projection_qtt_divergence_large_mu():
    """Through the QTT sweep, a large penalty leaves |G v| <= |G w| / (1 +
    mu h^2 lambda_min), lambda_min the smallest non-zero |g|^2."""
    n = 4
    X1, X2, dx = I.grid(n)
    ops = Q.build_operators(n, dx)
    w = [I.random_field(n, seed=42), I.random_field(n, seed=43)]
    wq = [Q.from_dense(f, 0.0, FULL) for f in w]
    h, mu = 1e-2, 1e9
    p = Q.Params(eps=0.0, chi_max=FULL, mu=mu, cg_tol=1e-14, cg_maxit=5000,
                 sweep_tol=1e-15, max_sweeps=60)
    v, _ = Q.project(wq, h, p, ops)
    vd = [Q.to_dense(x) for x in v]
    lam_min = (math.sin(2 * math.pi / 2 ** n) / dx) ** 2
    assert np.linalg.norm(Dn.divergence(vd, dx)) <= np.linalg.norm(Dn.divergence(w, dx)) / (
        1 + mu * h * h * lam_min) * 1.01


# ------------------------------------------------------------- RK4
def test_rk4_table_is_classical_rk4():
    """With no penalty the four Euler stages of Table RK4 / Eqs. U1-U4 sum
    to the classical RK4 update u + dt/6 (k1 + 2 k2 + 2 k3 + k4)."""
    n = 4
    _, _, dx = I.grid(n)
    u = [I.random_field(n, seed=50), I.random_field(n, seed=51)]
    dt, nu = 1e-2, 0.05
    f = lambda x: [-b for b in Dn.rhs_B(x, nu, dx)]
    k1 = f(u)
    k2 = f([u[i] + dt / 2 * k1[i] for i in range(2)])
    k3 = f([u[i] + dt / 2 * k2[i] for i in range(2)])
    k4 = f([u[i] + dt * k3[i] for i in range(2)])
    ref = [u[i] + dt / 6 * (k1[i] + 2 * k2[i] + 2 * k3[i] + k4[i]) for i in range(2)]
    out = Dn.rk4_step(u, dt, nu, 0.0, dx)
    for i in range(2):
        assert rel(out[i], ref[i]) < 1e-14


def test_qtt_rk4_equals_dense_rk4():
    """Untruncated QTT RK4 step == dense projected RK4 step."""
    n = 4
    X1, X2, dx = I.grid(n)
    ops = Q.build_operators(n, dx)
    u0, _ = I.taylor_green(n)
    u = [u0[0] + 0.1 * I.random_field(n, seed=3), u0[1] + 0.1 * I.random_field(n, seed=4)]
    uq = [Q.from_dense(f, 0.0, FULL) for f in u]
    p = Q.Params(eps=0.0, chi_max=FULL, **TIGHT)
    out = Q.rk4_step(uq, 1e-2, 0.01, p, ops)
    ref = Dn.rk4_step(u, 1e-2, 0.01, p.mu, dx)
    for i in range(2):
        assert rel(Q.to_dense(out[i]), ref[i]) < 1e-10


def test_taylor_green_closed_form_decay():
    """Taylor-Green (n = 6, nu = 0.01, dt = 1e-3, 10 steps) on the dense
    scheme: with the penalty strong enough to remove the pressure-like
    k = 2 residue, the TG amplitude decays as exp(-2 nu c^2 t),
    c = sin(dx)/dx the discrete symbol of the central difference (the
    continuum exp(-2 nu t) differs by 6.4e-7 at t = 0.01)."""
    n, nu, dt, steps = 6, 0.01, 1e-3, 10
    u0, dx = I.taylor_green(n)
    c2 = (math.sin(dx) / dx) ** 2
    T = steps * dt
    norm0 = sum(np.vdot(x, x) for x in u0)
    amp = lambda u: sum(np.vdot(u[i], u0[i]) for i in range(2)) / norm0
    v = [x.copy() for x in u0]
    for _ in range(steps):
        v = Dn.rk4_step(v, dt, nu, 1e12, dx)
    assert abs(amp(v) / math.exp(-2 * nu * c2 * T) - 1) < 1e-9
    assert abs(amp(v) / math.exp(-2 * nu * T) - 1) > 5e-7


def test_qtt_taylor_green_matches_dense():
    """The QTT oracle on the Taylor-Green problem (n = 6, eps = 1e-12, the
    paper's mu, two RK4 steps) reproduces the dense scheme, which the test
    above pins to the closed form."""
    n, nu, dt = 6, 0.01, 1e-3
    u0, dx = I.taylor_green(n)
    ops = Q.build_operators(n, dx)
    p = Q.Params(eps=1e-12, chi_max=64, cg_tol=1e-13, cg_maxit=2000, sweep_tol=1e-13)
    uq = [Q.from_dense(f, 1e-12, 64) for f in u0]
    v = [x.copy() for x in u0]
    for _ in range(2):
        uq = Q.rk4_step(uq, dt, nu, p, ops)
        v = Dn.rk4_step(v, dt, nu, p.mu, dx)
    for i in range(2):
        assert rel(Q.to_dense(uq[i]), v[i]) < 1e-10


def test_kinetic_energy_monotone():
    """Semi-discretely dE/dt = -nu sum |D_j u_i|^2 <= 0, convection is
    energy neutral and the projection a contraction: E never grows
    (Taylor-Green, n = 6, chi = 16, the paper's mu, QTT oracle)."""
    n, nu, dt = 6, 0.01, 1e-3
    u0, dx = I.taylor_green(n)
    ops = Q.build_operators(n, dx)
    p = Q.Params(eps=1e-12, chi_max=16, cg_tol=1e-12, cg_maxit=500, sweep_tol=1e-12)
    uq = [Q.from_dense(f, 1e-12, 16) for f in u0]
    E = [sum(Q.norm2(x) for x in uq)]
    for _ in range(4):
        uq = Q.rk4_step(uq, dt, nu, p, ops)
        E.append(sum(Q.norm2(x) for x in uq))
    assert all(E[k + 1] <= E[k] * (1 + 1e-14) for k in range(len(E) - 1))
    assert E[-1] < E[0]


# ------------------------------------------------------------- inputs
def test_initial_conditions_are_discretely_divergence_free():
    for gen in (lambda: I.shear_jet(7, seed=0), lambda: I.decaying_turbulence(7, k0=10, seed=0)):
        u, dx = gen()
        div = Dn.divergence(u, dx)
        assert np.abs(div).max() < 1e-10 * max(np.abs(Dn.d(u[0], 1, dx)).max(), 1.0)
    u, dx = I.decaying_turbulence(7, seed=1)
    assert abs(0.5 * np.mean(u[0] ** 2 + u[1] ** 2) - 1.0) < 1e-12


def test_qtt_euler_and_rk2_equal_dense():
    """Untruncated QTT Euler and midpoint-RK2 steps == the dense projected
    schemes (App. B: Eq. "euler"; Eqs. "midpoint_calc", "full_calc")."""
    n = 4
    X1, X2, dx = I.grid(n)
    ops = Q.build_operators(n, dx)
    u0, _ = I.taylor_green(n)
    u = [u0[0] + 0.1 * I.random_field(n, seed=5), u0[1] + 0.1 * I.random_field(n, seed=6)]
    uq = [Q.from_dense(f, 0.0, FULL) for f in u]
    p = Q.Params(eps=0.0, chi_max=FULL, **TIGHT)
    for qstep, dstep in ((Q.euler_step, Dn.euler_step), (Q.rk2_step, Dn.rk2_step)):
        out = qstep(uq, 1e-2, 0.01, p, ops)
        ref = dstep(u, 1e-2, 0.01, p.mu, dx)
        for i in range(2):
            assert rel(Q.to_dense(out[i]), ref[i]) < 1e-10


def test_euler_rk2_amplification_factors():
    """On the Taylor-Green mode the convection is energy-neutral and, with a
    strong penalty, the pressure part is projected out, so one step
    multiplies the mode amplitude by the scheme's amplification factor for
    y' = -lam y, lam = 2 nu c^2: 1 - lam dt (Euler), 1 - lam dt + (lam dt)^2 / 2
    (midpoint RK2), the Taylor polynomial of order 4 (RK4)."""
    n, nu, dt, steps = 6, 0.1, 1e-2, 10
    u0, dx = I.taylor_green(n)
    lam = 2 * nu * (math.sin(dx) / dx) ** 2
    z = lam * dt
    norm0 = sum(np.vdot(x, x) for x in u0)
    amp = lambda u: sum(np.vdot(u[i], u0[i]) for i in range(2)) / norm0
    factors = {Dn.euler_step: 1 - z, Dn.rk2_step: 1 - z + z * z / 2,
               Dn.rk4_step: 1 - z + z * z / 2 - z ** 3 / 6 + z ** 4 / 24}
    for step, g in factors.items():
        v = [x.copy() for x in u0]
        for _ in range(steps):
            v = step(v, dt, nu, 1e12, dx)
        assert abs(amp(v) / g ** steps - 1) < 1e-9, step.__name__
    # the three schemes are told apart at this step size
    assert abs((1 - z) ** steps / (1 - z + z * z / 2) ** steps - 1) > 1e-5


# ------------------------------------------------ higher-order stencils (Sec. II.B, App. D)
# Textbook central-difference weights c_1..c_m of orders 4, 6, 8 (from the
# Taylor conditions; e.g. Fornberg 1988, Table 1), typed in as the pin of
# the oracle's linear solve.
TEXTBOOK_WEIGHTS = {2: [1 / 2], 4: [2 / 3, -1 / 12], 6: [3 / 4, -3 / 20, 1 / 60],
                    8: [4 / 5, -1 / 5, 4 / 105, -1 / 280]}


def test_central_weights_textbook():
    for order, want in TEXTBOOK_WEIGHTS.items():
        np.testing.assert_allclose(Q.central_weights(order), want, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("a", [-5, -3, -1, 1, 2, 7])
@pytest.mark.parametrize("axis", [1, 2])
def test_shift_mpo_is_a_periodic_translation(a, axis):
    """S^a: every row of the dense MPO holds one 1 at the translated point."""
    n = 4
    N = 2 ** n
    M = Q.mpo_to_dense(Q.mpo_shift(n, axis, a))
    S = np.zeros((N * N, N * N))
    for x1 in range(N):
        for x2 in range(N):
            t = ((x1 + a) % N) * N + x2 if axis == 1 else x1 * N + (x2 + a) % N
            S[x1 * N + x2, t] = 1.0
    np.testing.assert_array_equal(M, S)


def test_order2_machine_equals_paper_carry_table():
    n = 5
    dx = 2 * math.pi / 2 ** n
    for axis in (1, 2):
        A = Q.mpo_to_dense(Q.mpo_diff_order(n, axis, dx, 2))
        B = Q.mpo_to_dense(Q.mpo_diff(n, axis, dx))
        assert np.abs(A - B).max() <= 1e-13 / dx


@pytest.mark.parametrize("order", [4, 6, 8])
@pytest.mark.parametrize("axis", [1, 2])
def test_high_order_diff_equals_stencil_bruteforce(order, axis):
    """Dense matrix of the order-p MPO == the periodic stencil with the
    textbook weights; D^T = -D."""
    n = 4
    N = 2 ** n
    dx = 2 * math.pi / N
    M = Q.mpo_to_dense(Q.mpo_diff_order(n, axis, dx, order))
    S = np.zeros((N * N, N * N))
    for x1 in range(N):
        for x2 in range(N):
            r = x1 * N + x2
            for k, c in enumerate(TEXTBOOK_WEIGHTS[order], start=1):
                for sgn in (1, -1):
                    t = (((x1 + sgn * k) % N) * N + x2 if axis == 1
                         else x1 * N + (x2 + sgn * k) % N)
                    S[r, t] += sgn * c / dx
    assert np.abs(M - S).max() <= 1e-12 / dx
    assert np.abs(M + M.T).max() <= 1e-12 / dx
    assert max(w.shape[3] for w in Q.mpo_diff_order(n, axis, dx, order)) <= 5


@pytest.mark.parametrize("order", [2, 4, 6, 8])
def test_high_order_diff_convergence_rate(order):
    """D sin(x) -> cos(x) with error ~ dx^order (closed form of the symbol
    sum_k 2 c_k sin(k dx) / dx), checked through the QTT at n = 5 and 6."""
    errs = []
    for n in (5, 6):
        X1, X2, dx = I.grid(n)
        D = Q.mpo_diff_order(n, 1, dx, order)
        q = Q.from_dense(np.sin(X1) * np.cos(X2), 1e-14, 64)
        out = Q.to_dense(Q.apply_mpo(D, q, 0.0, FULL))
        sym = sum(2 * c * math.sin(k * dx) for k, c in
                  enumerate(TEXTBOOK_WEIGHTS[order], start=1)) / dx
        assert rel(out, sym * np.cos(X1) * np.cos(X2)) < 1e-12
        errs.append(abs(sym - 1.0))
    rate = math.log2(errs[0] / errs[1])
    assert abs(rate - order) < 0.1, rate


def test_qtt_rk4_order4_equals_dense_rk4():
    """Untruncated QTT RK4 step with 4th-order stencils == the dense
    projected RK4 step with the same stencils (Fourier-space projection
    with the 4th-order symbols)."""
    n = 4
    X1, X2, dx = I.grid(n)
    ops = Q.build_operators(n, dx, order=4)
    u0, _ = I.taylor_green(n)
    u = [u0[0] + 0.1 * I.random_field(n, seed=3), u0[1] + 0.1 * I.random_field(n, seed=4)]
    uq = [Q.from_dense(f, 0.0, FULL) for f in u]
    p = Q.Params(eps=0.0, chi_max=FULL, **TIGHT)
    out = Q.rk4_step(uq, 1e-2, 0.01, p, ops)
    ref = Dn.rk4_step(u, 1e-2, 0.01, p.mu, dx, order=4)
    for i in range(2):
        assert rel(Q.to_dense(out[i]), ref[i]) < 1e-10


# ------------------------------------------------ TKE spectrum (Sec. III.A)
def test_tke_spectrum_parseval_and_single_modes():
    """Parseval: the shells of all wavevectors sum to 1/2 mean(u^2 + v^2);
    a single Fourier mode puts all its energy in the shell of its
    wavenumber; Taylor-Green (modes (+-1, +-1)) sits in shell round(sqrt 2) = 1."""
    n = 5
    N = 2 ** n
    X1, X2, dx = I.grid(n)
    u = [I.white_field(n, seed=1), I.white_field(n, seed=2)]
    kmax = int(math.ceil(math.sqrt(2) * N / 2)) + 1
    E = Dn.tke_spectrum(u, kmax)
    ke = 0.5 * np.mean(u[0] ** 2 + u[1] ** 2)
    assert abs(E.sum() - ke) <= 1e-13 * ke
    for (a, b, k) in ((3, 4, 5), (0, 7, 7), (5, 5, 7), (2, 1, 2)):
        f = np.cos(a * X1 + b * X2)
        E = Dn.tke_spectrum([f, np.zeros_like(f)], kmax)
        assert abs(E[k] - 0.25) < 1e-13 and abs(E.sum() - 0.25) < 1e-13, (a, b)
    tg, _ = I.taylor_green(n)
    E = Dn.tke_spectrum(tg, kmax)
    assert abs(E[1] - 0.25) < 1e-13 and abs(E.sum() - 0.25) < 1e-13


# ------------------------------------------------ the paper's implicit right-hand side (f1)
def test_hadamard_mpo_is_the_elementwise_product():
    n = 4
    A = Q.from_dense(I.random_field(n, seed=1), 0.0, FULL)
    B = Q.from_dense(I.random_field(n, seed=2), 0.0, FULL)
    out = Q.to_dense(Q.apply_mpo_exact(Q.hadamard_mpo(A), B))
    assert rel(out, Q.to_dense(A) * Q.to_dense(B)) < 1e-13


def test_implicit_projection_equals_fourier_solve():
    """At full rank the projection of the implicit right-hand side
    a u - h B(b) (never formed as an MPS) is the exact minimiser: the dense
    Fourier-space solve of w = a u - h B(b) computed densely (App. B)."""
    n = 4
    X1, X2, dx = I.grid(n)
    ops = Q.build_operators(n, dx)
    u0, _ = I.taylor_green(n)
    u = [u0[0] + 0.1 * I.random_field(n, seed=3), u0[1] + 0.1 * I.random_field(n, seed=4)]
    b = [u[0] + 0.05 * I.random_field(n, seed=5), u[1] - 0.05 * I.random_field(n, seed=6)]
    h, nu = 2e-2, 0.01
    p = Q.Params(eps=0.0, chi_max=FULL, **TIGHT)
    uq = [Q.from_dense(f, 0.0, FULL) for f in u]
    bq = [Q.from_dense(f, 0.0, FULL) for f in b]
    terms = Q.implicit_terms(uq, bq, h, nu, ops, 0.25)
    v, info = Q.project_implicit(terms, [Q.scaled(x, 0.25) for x in uq], h, p, ops)
    B = Dn.rhs_B(b, nu, dx)
    want = Dn.project([0.25 * u[i] - h * B[i] for i in range(2)], h, p.mu, dx)
    for i in range(2):
        assert rel(Q.to_dense(v[i]), want[i]) < 1e-10
    assert info.converged


def test_implicit_rk4_equals_dense_and_explicit():
    """Untruncated: the paper's form of the RK4 step equals the dense
    projected RK4 step and the explicit (B formed) QTT step."""
    n = 4
    X1, X2, dx = I.grid(n)
    ops = Q.build_operators(n, dx)
    u0, _ = I.taylor_green(n)
    u = [u0[0] + 0.1 * I.random_field(n, seed=3), u0[1] + 0.1 * I.random_field(n, seed=4)]
    uq = [Q.from_dense(f, 0.0, FULL) for f in u]
    p = Q.Params(eps=0.0, chi_max=FULL, **TIGHT)
    imp = Q.rk4_step_implicit(uq, 1e-2, 0.01, p, ops)
    ref = Dn.rk4_step(u, 1e-2, 0.01, p.mu, dx)
    exp_ = Q.rk4_step(uq, 1e-2, 0.01, p, ops)
    for i in range(2):
        assert rel(Q.to_dense(imp[i]), ref[i]) < 1e-10
        assert rel(Q.to_dense(imp[i]), Q.to_dense(exp_[i])) < 1e-10


# ------------------------------------------- exact spectral projection
@pytest.mark.parametrize("order", [2, 4, 8])
def test_exact_projection_invariants(order):
    """The exact projection (the mu -> infinity limit of the penalty solve)
    is checked in real space, not through its own Fourier formula: the
    result has zero discrete divergence under the stencil of `Dn.d`, the
    removed part is orthogonal to it, applying it twice changes nothing,
    and a discrete gradient (D_1 phi, D_2 phi) is removed entirely."""
    n = 5
    _, _, dx = I.grid(n)
    w = [I.white_field(n, seed=60), I.white_field(n, seed=61)]
    v = Dn.project_exact(w, dx, order)
    assert np.linalg.norm(Dn.divergence(v, dx, order)) < 1e-13 * np.linalg.norm(
        Dn.divergence(w, dx, order))
    r = [w[i] - v[i] for i in range(2)]
    assert abs(sum(np.vdot(r[i], v[i]) for i in range(2))) < 1e-13 * sum(
        np.vdot(x, x) for x in w)
    vv = Dn.project_exact(v, dx, order)
    for i in range(2):
        assert rel(vv[i], v[i]) < 1e-14
    phi = I.white_field(n, seed=62)
    grad = [Dn.d(phi, 1, dx, order), Dn.d(phi, 2, dx, order)]
    pg = Dn.project_exact(grad, dx, order)
    assert max(np.abs(x).max() for x in pg) < 1e-12 * max(np.abs(x).max() for x in grad)


def test_exact_projection_keeps_annihilated_modes():
    """Fields the central difference annihilates (a constant, and the
    alternating (-1)^x1 and (-1)^x2 patterns of the Nyquist modes) are
    divergence-free and pass unchanged; a divergence-free Taylor-Green field
    too.  A formula that took the rounding residue of sin(pi) as a non-zero
    symbol would zero the Nyquist mode of u_1."""
    n = 5
    N = 2 ** n
    _, _, dx = I.grid(n)
    alt = np.where(np.arange(N) % 2 == 0, 1.0, -1.0)
    w = [np.outer(alt, np.ones(N)) + 0.5, np.outer(np.ones(N), alt) - 0.25]
    for i, x in enumerate(Dn.project_exact(w, dx)):
        np.testing.assert_allclose(x, w[i], atol=1e-14)
    tg, dxt = I.taylor_green(n)
    for i, x in enumerate(Dn.project_exact(tg, dxt)):
        assert rel(x, tg[i]) < 1e-14


def test_exact_projection_is_the_penalty_limit():
    """|project(w, h, mu) - project_exact(w)| <= |w| / (1 + mu h^2 lambda_min)
    with lambda_min the smallest non-zero |g|^2 (the penalty solve damps
    each mode's divergent part by 1 / (1 + mu h^2 |g|^2))."""
    n = 5
    _, _, dx = I.grid(n)
    w = [I.white_field(n, seed=63), I.white_field(n, seed=64)]
    ve = Dn.project_exact(w, dx)
    lam_min = (math.sin(2 * math.pi / 2 ** n) / dx) ** 2
    nw = math.sqrt(sum(np.vdot(x, x) for x in w))
    for mu_h2 in (1e2, 1e6):
        vp = Dn.project(w, 1.0, mu_h2, dx)
        d = math.sqrt(sum(np.vdot(vp[i] - ve[i], vp[i] - ve[i]) for i in range(2)))
        assert d <= nw / (1 + mu_h2 * lam_min) * (1 + 1e-9)
        assert d >= 1e-3 * nw / (1 + mu_h2 * lam_min)  # the bound is not vacuous


def test_taylor_green_exact_projection_rk4_amplification():
    """With the exact projection the Taylor-Green convection term (a
    discrete gradient) is removed completely, so one RK4 step multiplies the
    field by the classical RK4 amplification 1 + z + z^2/2 + z^3/6 + z^4/24
    of the viscous decay, z = -2 nu c^2 dt, c = sin(dx)/dx."""
    n, nu, dt = 6, 0.01, 1e-3
    u0, dx = I.taylor_green(n)
    z = -2 * nu * (math.sin(dx) / dx) ** 2 * dt
    R = 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24
    v = Dn.rk4_step(u0, dt, nu, 0.0, dx, exact=True)
    for i in range(2):
        np.testing.assert_allclose(v[i], R * u0[i], atol=1e-14)


def test_qtt_spectral_projection_and_rk4_equal_dense():
    """The QTT oracle's spectral projection and its RK4 step with it
    (untruncated) reproduce the dense exact projection and the dense RK4
    step with exact projections; truncated to (eps, chi) the projection's
    result stays within the TT-SVD bound sqrt(n - 1) eps of the dense one."""
    n = 5
    _, _, dx = I.grid(n)
    ops = Q.build_operators(n, dx)
    u0, _ = I.taylor_green(n)
    u = [u0[0] + 0.1 * I.random_field(n, seed=65), u0[1] + 0.1 * I.random_field(n, seed=66)]
    uq = [Q.from_dense(f, 0.0, FULL) for f in u]
    p = Q.Params(eps=0.0, chi_max=FULL, projection="spectral")
    v, _ = Q.project_spectral(uq, p, ops)
    ve = Dn.project_exact(u, dx)
    for i in range(2):
        assert rel(Q.to_dense(v[i]), ve[i]) < 1e-13
    out = Q.rk4_step(uq, 1e-2, 0.01, p, ops)
    ref = Dn.rk4_step(u, 1e-2, 0.01, 0.0, dx, exact=True)
    for i in range(2):
        assert rel(Q.to_dense(out[i]), ref[i]) < 1e-12
    eps = 1e-3
    vt, _ = Q.project_spectral(uq, Q.Params(eps=eps, chi_max=FULL), ops)
    for i in range(2):
        assert rel(Q.to_dense(vt[i]), ve[i]) <= math.sqrt(n - 1) * eps


def test_qtt_euler_and_rk2_spectral_equal_dense():
    """Untruncated QTT Euler and midpoint RK2 steps with the spectral
    projection equal the dense steps built from the exact projection:
    P(u - dt B(u)) and P(u - dt B(P(u - dt/2 B(u))))."""
    n, dt, nu = 4, 1e-2, 0.02
    _, _, dx = I.grid(n)
    ops = Q.build_operators(n, dx)
    u = [I.random_field(n, seed=70), I.random_field(n, seed=71)]
    uq = [Q.from_dense(f, 0.0, FULL) for f in u]
    p = Q.Params(eps=0.0, chi_max=FULL, projection="spectral")
    B = Dn.rhs_B(u, nu, dx)
    e_ref = Dn.project_exact([u[i] - dt * B[i] for i in range(2)], dx)
    um = Dn.project_exact([u[i] - 0.5 * dt * B[i] for i in range(2)], dx)
    Bm = Dn.rhs_B(um, nu, dx)
    r_ref = Dn.project_exact([u[i] - dt * Bm[i] for i in range(2)], dx)
    e = Q.euler_step(uq, dt, nu, p, ops)
    r = Q.rk2_step(uq, dt, nu, p, ops)
    for i in range(2):
        assert rel(Q.to_dense(e[i]), e_ref[i]) < 1e-12
        assert rel(Q.to_dense(r[i]), r_ref[i]) < 1e-12
