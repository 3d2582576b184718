"""Diagnostics on the GPU: the MPS inner product against the oracle's
transfer matrices, and the closed forms it must reproduce (the Taylor-Green
kinetic energy 1/4, the fidelity of a state with itself and with a scaled
copy)."""
import numpy as np
import pytest

import qtt_inputs as I
from oracle import qtt as Q

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2406_17823_b300 as P
    return P


def test_inner_matches_oracle(P):
    n = 6
    ctx = P.Context(n)
    A = I.random_cores(n, [1, 4, 16, 33, 16, 4, 1], seed=11)
    B = I.random_cores(n, [1, 3, 9, 20, 12, 4, 1], seed=12)
    got = ctx.inner(ctx.from_cores(A), ctx.from_cores(B))
    want = Q.inner(A, B)
    assert abs(got - want) <= 1e-12 * max(1.0, abs(want))
    # and the dense definition
    dense = float(np.sum(Q.to_dense(A) * Q.to_dense(B)))
    assert abs(got - dense) <= 1e-11 * max(1.0, abs(dense))


def test_taylor_green_energy_and_fidelity(P):
    n = 6
    ctx = P.Context(n)
    (u, v), dx = I.taylor_green(n)
    a, b = ctx.from_dense(u), ctx.from_dense(v)
    assert abs(ctx.kinetic_energy(a, b) - 0.25) < 1e-13
    assert abs(ctx.fidelity(a, a) - 1.0) < 1e-13
    c = ctx.add([-3.0], [a])
    assert abs(ctx.fidelity(a, c) - 1.0) < 1e-13
    assert ctx.fidelity(a, b) < 1e-20  # sin x cos y and cos x sin y are orthogonal


@pytest.mark.parametrize("n", [5, 10])
def test_tke_spectrum_matches_oracle(P, n):
    """The TKE spectrum on the device (dense readout, own FFTs, shell sums)
    against the oracle's numpy-FFT spectrum of the same fields, element by
    element, and Parseval against the kinetic energy of the QTT."""
    from oracle import dense as Dn
    ctx = P.Context(n, eps=1e-8, chi_max=64)
    (u, v), dx = I.shear_jet(n, seed=0) if n >= 7 else I.taylor_green(n)
    if n < 7:
        u = u + 0.1 * I.white_field(n, seed=4)
    a, b = ctx.from_dense(u), ctx.from_dense(v)
    kmax = int(np.ceil(2 ** n / np.sqrt(2.0))) + 1
    got = ctx.tke_spectrum(a, b, kmax)
    want = Dn.tke_spectrum([ctx.to_dense(a).cpu().numpy(), ctx.to_dense(b).cpu().numpy()], kmax)
    assert np.all(np.abs(got - want) <= 1e-12 * want.sum())
    big = want > 1e-6 * want.max()
    assert np.max(np.abs(got[big] - want[big]) / want[big]) < 1e-9
    assert abs(got.sum() - ctx.kinetic_energy(a, b)) <= 1e-12 * got.sum()
    # a truncated shell range leaves the rest out
    assert np.array_equal(ctx.tke_spectrum(a, b, 3), got[:4])


def test_tke_spectrum_taylor_green_shell(P):
    """Taylor-Green sits in shell round(sqrt 2) = 1 with energy 1/4."""
    n = 6
    ctx = P.Context(n)
    (u, v), dx = I.taylor_green(n)
    E = ctx.tke_spectrum(ctx.from_dense(u), ctx.from_dense(v), 10)
    assert abs(E[1] - 0.25) < 1e-13 and abs(E.sum() - 0.25) < 1e-13
