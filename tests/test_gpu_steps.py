"""The lower-order steps of App. B on the GPU against the oracle: explicit
Euler (Eq. "euler") and the midpoint RK2 (Eqs. "midpoint_calc",
"full_calc"), one step each from a perturbed Taylor-Green field and from a
small shear jet, 1e-10 relative L2 on the dense fields."""
import numpy as np
import pytest

import qtt_inputs as I
from oracle import qtt as Q

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2406_17823_b300 as P
    return P


def cases():
    n = 5
    u0, dx = I.taylor_green(n)
    tg = [u0[0] + 0.05 * I.random_field(n, seed=1), u0[1]]
    (ju, jv), jdx = I.shear_jet(6, seed=2)
    return [("taylor_green_n5", 5, tg, dx, 1e-3, 0.01,
             dict(eps=1e-12, chi_max=16, cg_tol=1e-12, cg_maxit=500, sweep_tol=1e-12)),
            ("shear_jet_n6", 6, [ju, jv], jdx, 0.1 * jdx / float(np.abs(ju).max()), 1e-3,
             dict(eps=1e-8, chi_max=12))]


@pytest.mark.parametrize("which", ["euler", "rk2"])
@pytest.mark.parametrize("case", range(2))
def test_step_parity(P, which, case):
    name, n, u, dx, dt, nu, pp = cases()[case]
    ctx = P.Context(n, **pp)
    uq = [Q.from_dense(f, pp["eps"], pp["chi_max"]) for f in u]
    g = [ctx.from_cores(c) for c in uq]
    getattr(ctx, f"{which}_step")(g[0], g[1], dt, nu)
    ops = Q.build_operators(n, dx)
    ref = getattr(Q, f"{which}_step")(uq, dt, nu, Q.Params(**pp), ops)
    for i in range(2):
        got = ctx.to_dense(g[i]).cpu().numpy()
        want = Q.to_dense(ref[i])
        assert np.linalg.norm(got - want) <= 1e-10 * np.linalg.norm(want), name
