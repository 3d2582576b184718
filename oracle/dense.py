"""Dense small-grid reference: the plain definition the QTT scheme approximates.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The same discrete scheme as the QTT method, with no tensor network and no
truncation: fields are dense N x N arrays (axis 0 = x1, axis 1 = x2), the
central difference is a periodic stencil (Eq. "fdm"), products are
element-wise, and the penalty projection (I + mu h^2 G^T G) v = w with
G = [D_1 D_2] is solved exactly per Fourier mode.
"""
from __future__ import annotations

import numpy as np


def _weights(order: int):
    """Central-difference weights c_1..c_m of the given even order (the
    same conditions as oracle.qtt.central_weights)."""
    from oracle.qtt import central_weights
    return central_weights(order)


def d(F: np.ndarray, axis: int, dx: float, order: int = 2) -> np.ndarray:
    """Central difference along axis 1 (x1) or 2 (x2), periodic: order 2 is
    (F(x+1) - F(x-1)) / (2 dx); order 2m is sum_k c_k (F(x+k) - F(x-k)) / dx."""
    ax = axis - 1
    if order == 2:
        return (np.roll(F, -1, axis=ax) - np.roll(F, 1, axis=ax)) / (2.0 * dx)
    out = np.zeros_like(F)
    for k, c in enumerate(_weights(order), start=1):
        out += c * (np.roll(F, -k, axis=ax) - np.roll(F, k, axis=ax))
    return out / dx


def convection(u, dx, order: int = 2):
    """Skew-symmetric convection 1/2 sum_j (u_j D_j u_i + D_j(u_j u_i)) (App. B)."""
    out = []
    for i in range(2):
        acc = np.zeros_like(u[i])
        for j in range(2):
            acc += 0.5 * (u[j] * d(u[i], j + 1, dx, order) + d(u[j] * u[i], j + 1, dx, order))
        out.append(acc)
    return out


def rhs_B(u, nu, dx, order: int = 2):
    """B_i = convection_i - nu sum_j D_j D_j u_i (App. B, Eq. for B_i)."""
    conv = convection(u, dx, order)
    return [conv[i] - nu * sum(d(d(u[i], j, dx, order), j, dx, order) for j in (1, 2))
            for i in range(2)]


def symbols(N: int, dx: float, order: int = 2):
    """Fourier symbols g_j of D_j (axis 0, 1): i sin(2 pi m_j / N) / dx for
    order 2, i sum_k 2 c_k sin(2 pi k m_j / N) / dx for order 2m."""
    m = np.fft.fftfreq(N) * N
    if order == 2:
        g = 1j * np.sin(2.0 * np.pi * m / N) / dx
    else:
        g = 1j * sum(2.0 * c * np.sin(2.0 * np.pi * k * m / N)
                     for k, c in enumerate(_weights(order), start=1)) / dx
    return g[:, None] * np.ones((1, N)), np.ones((N, 1)) * g[None, :]


def project(w, h: float, mu: float, dx: float, order: int = 2):
    """Exact minimiser of mu |D1 v1 + D2 v2|^2 + |v - w|^2 / h^2.

    Per Fourier mode the normal matrix is I + c conj(g) g^T (c = mu h^2;
    D_j^T = -D_j has symbol conj(g_j)); Sherman-Morrison gives
    v = w - c conj(g) (g^T w) / (1 + c |g|^2).
    """
    N = w[0].shape[0]
    g1, g2 = symbols(N, dx, order)
    c = mu * h * h
    W1, W2 = np.fft.fft2(w[0]), np.fft.fft2(w[1])
    gw = g1 * W1 + g2 * W2
    den = 1.0 + c * (np.abs(g1) ** 2 + np.abs(g2) ** 2)
    V1 = W1 - c * np.conj(g1) * gw / den
    V2 = W2 - c * np.conj(g2) * gw / den
    return [np.real(np.fft.ifft2(V1)), np.real(np.fft.ifft2(V2))]


def project_exact(w, dx: float, order: int = 2):
    """The exact discrete projection onto the kernel of G = [D_1 D_2]: the
    limit mu -> infinity of `project`, the alternative to the penalty that
    the paper's outlook (Sec. IV, periodic boundaries, Fourier transforms)
    points to.  Per Fourier mode g^T w is removed along conj(g):
    v = w - conj(g) (g^T w) / |g|^2; with g_j = i sigma_j (sigma_j real,
    D_j^T = -D_j) this is v = w - sigma (sigma . w) / |sigma|^2.  Modes
    where both symbols vanish (2 m_j = 0 mod N: the mean and the Nyquist
    modes, which every central difference annihilates) pass unchanged;
    there sigma_j is set to exactly zero instead of the rounding residue of
    sin(pi)."""
    N = w[0].shape[0]
    m = (np.fft.fftfreq(N) * N).astype(np.int64)
    if order == 2:
        sig = np.sin(2.0 * np.pi * m / N) / dx
    else:
        sig = sum(2.0 * c * np.sin(2.0 * np.pi * k * m / N)
                  for k, c in enumerate(_weights(order), start=1)) / dx
    sig[(2 * m) % N == 0] = 0.0
    s1, s2 = sig[:, None] * np.ones((1, N)), np.ones((N, 1)) * sig[None, :]
    W1, W2 = np.fft.fft2(w[0]), np.fft.fft2(w[1])
    den = s1 * s1 + s2 * s2
    t = np.where(den > 0, (s1 * W1 + s2 * W2) / np.where(den > 0, den, 1.0), 0.0)
    return [np.real(np.fft.ifft2(W1 - s1 * t)), np.real(np.fft.ifft2(W2 - s2 * t))]


def divergence(u, dx, order: int = 2):
    return d(u[0], 1, dx, order) + d(u[1], 2, dx, order)


RK4_H = (1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0)
RK4_B = (None, (3.0, 0.25), (1.5, 0.625), (3.0, 0.25))


def rk4_step(u, dt, nu, mu, dx, order: int = 2, exact: bool = False):
    """Four projected Euler stages (App. B, Table RK4, Eqs. U1-U4); with
    exact=True each stage takes the exact projection `project_exact`
    instead of the penalty solve."""
    U = []
    b = u
    for s in range(4):
        if s > 0:
            c1, c2 = RK4_B[s]
            b = [c1 * U[s - 1][i] + c2 * u[i] for i in range(2)]
        h = RK4_H[s] * dt
        B = rhs_B(b, nu, dx, order)
        w = [0.25 * u[i] - h * B[i] for i in range(2)]
        U.append(project_exact(w, dx, order) if exact else project(w, h, mu, dx, order))
    return [U[0][i] + U[1][i] + U[2][i] + U[3][i] for i in range(2)]


def euler_step(u, dt, nu, mu, dx):
    """Projected explicit Euler (App. B, Eq. "euler"): P(u - dt B(u))."""
    B = rhs_B(u, nu, dx)
    return project([u[i] - dt * B[i] for i in range(2)], dt, mu, dx)


def rk2_step(u, dt, nu, mu, dx):
    """Projected midpoint RK2 (App. B, Eqs. "midpoint_calc", "full_calc")."""
    B = rhs_B(u, nu, dx)
    um = project([u[i] - 0.5 * dt * B[i] for i in range(2)], 0.5 * dt, mu, dx)
    B = rhs_B(um, nu, dx)
    return project([u[i] - dt * B[i] for i in range(2)], dt, mu, dx)



def tke_spectrum(u, kmax: int):
    """Turbulent kinetic energy spectrum of a velocity field on the periodic
    N x N grid (Sec. III.A, the TKE spectra of the paper's figures):
    E(k) = sum over wavevectors (m1, m2) with round(|m|) = k of
    (|u_hat|^2 + |v_hat|^2) / (2 N^4), u_hat = fft2(u), k = 0..kmax (integer
    shells in units of the fundamental 2 pi / L; wavevectors beyond kmax
    are left out).  By Parseval sum_k E(k) = 1/2 mean(u^2 + v^2) when kmax
    covers every shell.  A shell holds the integers q = m1^2 + m2^2 with
    (k - 1/2)^2 < q < (k + 1/2)^2, i.e. k^2 - k + 1 <= q <= k^2 + k (q = 0 for
    k = 0): no wavevector sits on a shell boundary."""
    N = u[0].shape[0]
    P = sum(np.abs(np.fft.fft2(c)) ** 2 for c in u)
    m = (np.fft.fftfreq(N) * N).astype(np.int64)
    q = m[:, None] ** 2 + m[None, :] ** 2
    E = np.zeros(kmax + 1)
    for k in range(kmax + 1):
        sel = (q == 0) if k == 0 else ((q >= k * k - k + 1) & (q <= k * k + k))
        E[k] = P[sel].sum() / (2.0 * N ** 4)
    return E
