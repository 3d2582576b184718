"""The exact spectral projection on the GPU (qtt_project_spectral and
qtt_params.projection = QTT_PROJ_SPECTRAL): the alternative to the penalty
that the paper's outlook (Sec. IV) points to for periodic boundaries, the
orthogonal projection onto the kernel of the discrete divergence, computed
through 2-D FFTs on the device and re-encoded by TT-SVD.  Dense fields
against the oracle's project_spectral / rk4_step with projection "spectral"
(1e-10 FP64, 1e-6 mixed), the discrete divergence of the result against the
stencil, the Taylor-Green RK4 amplification in closed form, and whole-step
graphs bit for bit."""
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


def divergent_pair(n, seed):
    """A shear jet with a random smooth field added to v: not divergence-free."""
    (u, v), dx = I.shear_jet(n, delta=2 * math.pi / 60, seed=seed)
    return [u, v + 0.3 * I.random_field(n, seed=seed + 7)], dx


@pytest.mark.parametrize("prec,tol", [(0, TOL), (1, 1e-6)])
@pytest.mark.parametrize("n,eps,chi,order", [(6, 1e-10, 16, 2), (7, 1e-8, 32, 2),
                                             (7, 1e-8, 32, 8), (5, 0.0, 64, 4)])
def test_project_spectral_matches_oracle(P, n, eps, chi, order, prec, tol):
    w, dx = divergent_pair(n, seed=n)
    ctx = P.Context(n, eps=eps, chi_max=chi, fd_order=order, precision=prec)
    wq = [Q.from_dense(f, eps, chi) for f in w]
    g = [ctx.from_cores(c) for c in wq]
    v1, v2 = ctx.project_spectral(g[0], g[1])
    ops = Q.build_operators(n, dx, order)
    ref, _ = Q.project_spectral(wq, Q.Params(eps=eps, chi_max=chi), ops)
    got = [ctx.to_dense(x).cpu().numpy() for x in (v1, v2)]
    for i in range(2):
        assert rel(got[i], Q.to_dense(ref[i])) <= tol
    assert v1.bonds == Q.bond_dims(ref[0]) or prec == 1
    assert_divergence_from_encoding_only(wq, got, dx, order)


def assert_divergence_from_encoding_only(wq, got, dx, order=2):
    """The divergence left in the result is that of its re-encoding error d
    (v minus the exact projection of w): |G d| <= sqrt(2) sigma_max |d|,
    sigma_max <= sum_k 2|c_k| / dx the largest symbol of D_j."""
    wd = [Q.to_dense(x) for x in wq]
    exact = Dn.project_exact(wd, dx, order)
    div_in = np.linalg.norm(Dn.divergence(wd, dx, order))
    div_out = np.linalg.norm(Dn.divergence(got, dx, order))
    dn = math.sqrt(sum(float(np.sum((a - b) ** 2)) for a, b in zip(got, exact)))
    smax = 2 * float(np.abs(Q.central_weights(order)).sum()) / dx
    print(f"divergence {div_in:.3e} -> {div_out:.3e} (encoding error {dn:.3e})")
    assert div_out <= math.sqrt(2) * smax * dn * (1 + 1e-9) + 1e-12 * div_in


def test_project_spectral_full_size(P):
    """The bench's grid (2^10, chi 64, eps 1e-8): FP64 within 1e-10 of the
    oracle, the divergence left only the re-encoding's."""
    n, eps, chi = 10, 1e-8, 64
    w, dx = divergent_pair(n, seed=3)
    ctx = P.Context(n, eps=eps, chi_max=chi)
    wq = [Q.from_dense(f, eps, chi) for f in w]
    g = [ctx.from_cores(c) for c in wq]
    v1, v2 = ctx.project_spectral(g[0], g[1])
    ref, _ = Q.project_spectral(wq, Q.Params(eps=eps, chi_max=chi), Q.build_operators(n, dx))
    got = [ctx.to_dense(x).cpu().numpy() for x in (v1, v2)]
    for i in range(2):
        assert rel(got[i], Q.to_dense(ref[i])) <= TOL
    assert_divergence_from_encoding_only(wq, got, dx)


@pytest.mark.parametrize("prec,tol", [(0, TOL), (1, 1e-6)])
@pytest.mark.parametrize("n,chi", [(6, 16), (7, 32)])
def test_rk4_spectral_matches_oracle(P, n, chi, prec, tol):
    """One RK4 step of the shear jet with every stage projected exactly
    (explicit right-hand side, eps 1e-8): FP64 at 1e-10, mixed at 1e-6."""
    (u, v), dx = I.shear_jet(n, delta=2 * math.pi / 60, seed=0)
    dt, nu = 0.1 * dx / float(np.abs(u).max()), 1 / 2e5
    pp = dict(eps=1e-8, chi_max=chi)
    ctx = P.Context(n, precision=prec, projection=P.PROJ_SPECTRAL, **pp)
    uq = [Q.from_dense(f, pp["eps"], chi) for f in (u, v)]
    g = [ctx.from_cores(c) for c in uq]
    ref = Q.rk4_step(uq, dt, nu, Q.Params(projection="spectral", **pp),
                     Q.build_operators(n, dx))
    ctx.rk4_step(g[0], g[1], dt, nu)
    for i in range(2):
        assert rel(ctx.to_dense(g[i]).cpu().numpy(), Q.to_dense(ref[i])) <= tol


@pytest.mark.parametrize("which", ["euler", "rk2"])
def test_lower_order_steps_spectral(P, which):
    n = 6
    (u, v), dx = I.shear_jet(n, seed=2)
    dt, nu = 0.1 * dx / float(np.abs(u).max()), 1e-3
    pp = dict(eps=1e-8, chi_max=12)
    ctx = P.Context(n, projection=P.PROJ_SPECTRAL, **pp)
    uq = [Q.from_dense(f, pp["eps"], pp["chi_max"]) for f in (u, v)]
    g = [ctx.from_cores(c) for c in uq]
    getattr(ctx, f"{which}_step")(g[0], g[1], dt, nu)
    ref = getattr(Q, f"{which}_step")(uq, dt, nu, Q.Params(projection="spectral", **pp),
                                      Q.build_operators(n, dx))
    for i in range(2):
        assert rel(ctx.to_dense(g[i]).cpu().numpy(), Q.to_dense(ref[i])) <= TOL


def test_rk4_spectral_taylor_green_closed_form(P):
    """Taylor-Green at n = 6: the exact projection removes the convection
    term (a discrete gradient) entirely, so three RK4 steps multiply the field
    by R(z)^3, R the classical RK4 amplification of z = -2 nu c^2 dt,
    c = sin(dx)/dx."""
    n, nu, dt = 6, 0.01, 1e-3
    u0, dx = I.taylor_green(n)
    ctx = P.Context(n, eps=1e-12, chi_max=16, projection=P.PROJ_SPECTRAL)
    g = [ctx.from_dense(f) for f in u0]
    for _ in range(3):
        ctx.rk4_step(g[0], g[1], dt, nu)
    z = -2 * nu * (math.sin(dx) / dx) ** 2 * dt
    R = 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24
    for i in range(2):
        assert rel(ctx.to_dense(g[i]).cpu().numpy(), R ** 3 * u0[i]) <= 1e-11


@pytest.mark.parametrize("prec", [0, 1])
def test_spectral_step_graph_replays_bit_for_bit(P, prec):
    (u, v), dx = I.shear_jet(6, seed=2)
    dt, nu = 0.1 * dx / float(np.abs(u).max()), 1e-4
    out = []
    for graphs in (0, 2):
        ctx = P.Context(6, eps=1e-8, chi_max=16, graphs=graphs, projection=P.PROJ_SPECTRAL,
                        precision=prec)
        a, b = ctx.from_dense(u), ctx.from_dense(v)
        for _ in range(4):
            ctx.rk4_step(a, b, dt, nu)
        if graphs:
            assert ctx.graph_stats()[1] >= 2
        out.append([ctx.to_dense(a).cpu().numpy(), ctx.to_dense(b).cpu().numpy()])
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_spectral_rejected_with_implicit_rhs(P):
    with pytest.raises(P.QttError):
        P.Context(6, projection=P.PROJ_SPECTRAL, rhs_form=P.RHS_IMPLICIT)
