"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds no arithmetic of the time-stepping method itself: it
draws random numbers and evaluates closed-form initial conditions on the
grid.  Both the CUDA path (through its Python binding) and the CPU oracle
take their inputs from here and from nowhere else.

Grids are periodic, N = 2**n points per side over [0, L)^2, point
(x1, x2) at (x1 * dx, x2 * dx) with dx = L / N; arrays are indexed
F[x1, x2] (x1 slow), float64.
"""
from __future__ import annotations

import math

import numpy as np

TWO_PI = 2.0 * math.pi


def grid(n: int, L: float = TWO_PI):
    N = 2 ** n
    dx = L / N
    x = np.arange(N) * dx
    X1, X2 = np.meshgrid(x, x, indexing="ij")
    return X1, X2, dx


def taylor_green(n: int):
    """u = sin x cos y, v = -cos x sin y on [0, 2 pi)^2."""
    X1, X2, dx = grid(n)
    return [np.sin(X1) * np.cos(X2), -np.cos(X1) * np.sin(X2)], dx


def _stencil(F, axis, dx):
    ax = axis - 1
    return (np.roll(F, -1, axis=ax) - np.roll(F, 1, axis=ax)) / (2.0 * dx)


def _velocity_from_streamfunction(psi, dx):
    """u = d psi / d x2, v = -d psi / d x1 with the periodic central stencil,
    so that the stencil divergence of (u, v) vanishes identically."""
    return _stencil(psi, 2, dx), -_stencil(psi, 1, dx)


def shear_jet(n: int, delta: float = TWO_PI / 200.0, amp: float = 0.05,
              noise: float = 1e-3, seed: int = 0):
    """Double shear layer ("jet") on [0, 2 pi)^2.

    u = tanh((y - pi/2)/delta) - tanh((y - 3 pi/2)/delta),
    v = amp * sin(x), plus a seeded divergence-free perturbation whose
    per-component RMS is `noise` (white stream function differentiated by
    the central stencil).
    """
    X1, X2, dx = grid(n)
    u = np.tanh((X2 - 0.5 * math.pi) / delta) - np.tanh((X2 - 1.5 * math.pi) / delta)
    v = amp * np.sin(X1)
    if noise > 0.0:
        rng = np.random.default_rng(seed)
        psi = rng.standard_normal(u.shape)
        nu_, nv_ = _velocity_from_streamfunction(psi, dx)
        rms = math.sqrt(0.5 * (np.mean(nu_ ** 2) + np.mean(nv_ ** 2)))
        u = u + noise * nu_ / rms
        v = v + noise * nv_ / rms
    return [u, v], dx


def decaying_turbulence(n: int, k0: float = 10.0, seed: int = 0):
    """Random-phase 2-D turbulence with E(k) ~ k^4 exp(-2 (k/k0)^2).

    The vorticity amplitude per mode is sqrt(k E(k) / pi) with a uniform
    random phase; the real part of the inverse FFT is kept (which makes the
    spectrum Hermitian), the stream function solves -lap psi = omega
    spectrally, the velocity follows from psi by the central stencil, and
    the field is scaled to unit kinetic energy 1/2 mean(u^2 + v^2) = 1.
    """
    X1, X2, dx = grid(n)
    N = 2 ** n
    rng = np.random.default_rng(seed)
    m = np.fft.fftfreq(N) * N
    K1, K2 = np.meshgrid(m, m, indexing="ij")
    k = np.sqrt(K1 ** 2 + K2 ** 2)
    E = k ** 4 * np.exp(-2.0 * (k / k0) ** 2)
    amp = np.sqrt(k * E / math.pi)
    phase = rng.uniform(0.0, TWO_PI, size=k.shape)
    w_hat = amp * np.exp(1j * phase)
    k2 = np.where(k > 0, k ** 2, 1.0)
    psi_hat = np.where(k > 0, w_hat / k2, 0.0)
    psi = np.real(np.fft.ifft2(psi_hat))
    u, v = _velocity_from_streamfunction(psi, dx)
    ke = 0.5 * np.mean(u ** 2 + v ** 2)
    s = 1.0 / math.sqrt(ke) if ke > 0 else 1.0
    return [u * s, v * s], dx


def random_cores(n: int, bonds, seed: int = 0, scale: float = 1.0):
    """Seeded Gaussian MPS cores with the given bonds (len n+1, ends 1)."""
    rng = np.random.default_rng(seed)
    bonds = list(bonds)
    assert len(bonds) == n + 1 and bonds[0] == 1 and bonds[-1] == 1
    return [scale * rng.standard_normal((bonds[k], 4, bonds[k + 1])) for k in range(n)]


def natural_bonds(n: int, chi: int):
    """min(4^k, 4^(n-k), chi) for k = 0..n."""
    return [min(4 ** k, 4 ** (n - k), chi) for k in range(n + 1)]


def random_field(n: int, modes: int = 6, seed: int = 0):
    """A smooth seeded periodic field: a few random low Fourier modes."""
    X1, X2, _ = grid(n)
    rng = np.random.default_rng(seed)
    F = np.zeros_like(X1)
    for _ in range(modes):
        k1, k2 = rng.integers(-3, 4, size=2)
        a, ph = rng.standard_normal(), rng.uniform(0, TWO_PI)
        F += a * np.cos(k1 * X1 + k2 * X2 + ph)
    return F


def white_field(n: int, seed: int = 0):
    """Gaussian white-noise field (full QTT rank)."""
    return np.random.default_rng(seed).standard_normal((2 ** n, 2 ** n))
