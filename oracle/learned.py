"""Learned truncation: oracle of the randomised compression and of its MLP.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The plain method cuts every bond of the right-to-left compression sweep
with a full truncated SVD (Sec. II.C; per-bond epsilon rule of
:func:`oracle.qtt.trunc_rank`).  The learned form replaces that SVD, where a
predicted rank is available, by a randomised range finder (Halko, Martinsson
and Tropp, SIAM Review 53 (2011), Algorithm 4.1: Y = M Omega, Q = orth(Y),
B = Q^T M, SVD of the small B) of width w = predicted rank + oversampling.
The weight of M outside span(Q), |M|_F^2 - |B|_F^2 = |M - Q Q^T M|_F^2, is
the error estimate: when it exceeds ACCEPT eps^2 |M|_F^2 (ACCEPT = 0.1: the
sketch may miss at most a tenth of the bond's truncation budget) the bond falls
back to the full SVD; otherwise the eps rule runs on the singular values of
B with that outside weight counted as discarded, and chi_max caps the rank.  The
estimate is a difference of two sums of squares, so its rounding floor is
about 1e-16 |M|_F^2: the rule is meaningful for eps above about 1e-7 (the
learned form's workloads use eps = 1e-6).

The predicted rank comes from a two-layer perceptron (33 features -> 64 ReLU
units -> 1 output) fed with the previous step's spectrum at the same bond
(top 32 values of log10(sigma / sigma_1), clipped at -16 and scaled by 1/16)
and the bond index divided by n; its output times chi_max, rounded and
clipped to [1, chi_max], is the rank.  Training minimises the mean squared
error against rank / chi_max with Adam (Kingma and Ba, ICLR 2015).

Omega's entries come from a counter-based generator, so that any entry can
be produced independently on either side: SplitMix64 (Steele, Lea and Flood,
OOPSLA 2014) evaluated at state key + (i + 1) * 0x9E3779B97F4A7C15 gives 64
random bits for counter i; the top 53 bits give a uniform in (0, 1); two
uniforms give one standard normal by the Box-Muller transform (Box and
Muller 1958).  Entry (i, j) of Omega uses counters 2e and 2e + 1 with
e = i * 1024 + j, i the row index (s, b) -> s * D_k + b of the unfolding and
j < w the column; the key of a bond is (seed << 40) ^ (slot << 8) ^ bond.

parity: the generator is pinned by the published SplitMix64 output stream
and by moments; the range finder by the exact residual, by equality with
the full SVD when the range finder spans M, and by its fallback rule; the
perceptron's gradient by central differences (tests/test_oracle_learned.py).
"""
from __future__ import annotations

import numpy as np

from . import qtt as Q

GOLDEN = 0x9E3779B97F4A7C15
MASK = (1 << 64) - 1
N_FEAT = 33
N_HID = 64
N_PARAM = N_HID * N_FEAT + N_HID + N_HID + 1
OMEGA_STRIDE = 1024
ACCEPT = 0.1


# ------------------------------------------------------------ generator
def splitmix64(state: int) -> int:
    """SplitMix64 output for one state value (the mix of Steele et al.)."""
    z = state & MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def bits(key: int, i: int) -> int:
    """64 random bits for counter i under `key`."""
    return splitmix64((key + (i + 1) * GOLDEN) & MASK)


def uniform(key: int, i: int) -> float:
    return ((bits(key, i) >> 11) + 0.5) * 2.0 ** -53


def gaussian(key: int, e: int) -> float:
    u1, u2 = uniform(key, 2 * e), uniform(key, 2 * e + 1)
    return float(np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2))


def bond_key(seed: int, slot: int, bond: int) -> int:
    return ((seed << 40) ^ (slot << 8) ^ bond) & MASK


def omega(key: int, rows: int, w: int) -> np.ndarray:
    """Gaussian test matrix (rows x w), entry (i, j) from counter i*1024+j."""
    if w > OMEGA_STRIDE:
        raise ValueError("width above the generator's row stride")
    O = np.empty((rows, w))
    for i in range(rows):
        for j in range(w):
            O[i, j] = gaussian(key, i * OMEGA_STRIDE + j)
    return O


# ------------------------------------------------------ range finder
def range_finder(M: np.ndarray, w: int, key: int):
    """Algorithm 4.1 of Halko et al. for one unfolding M (D x N).

    Returns (Q, B, outside) with Q (D x w') orthonormal, B = Q^T M and
    outside = |M|_F^2 - |B|_F^2 (clipped at 0), w' = min(w, D, N).
    """
    D, N = M.shape
    w = min(w, D, N)
    Y = M @ omega(key, N, w)
    Qm, _ = np.linalg.qr(Y)
    B = Qm.T @ M
    outside = max(float(np.sum(M * M)) - float(np.sum(B * B)), 0.0)
    return Qm, B, outside


def trunc_rank_total(s: np.ndarray, extra: float, eps: float, chi_max: int) -> int:
    """:func:`oracle.qtt.trunc_rank` with `extra` weight outside the spectrum
    counted as discarded: the smallest r with sum_{j>r} s_j^2 + extra <=
    eps^2 (sum_j s_j^2 + extra), capped at chi_max."""
    s2 = np.asarray(s, dtype=np.float64) ** 2
    m = s2.shape[0]
    tail = np.zeros(m + 1)
    tail[m] = extra
    for j in range(m - 1, -1, -1):
        tail[j] = tail[j + 1] + s2[j]
    total = tail[0]
    if total == 0.0 or m == 0:
        return 1
    thr = eps * eps * total
    r = m
    for cand in range(1, m + 1):
        if tail[cand] <= thr:
            r = cand
            break
    return max(1, min(r, chi_max))


def compress_rf(cores: list, eps: float, chi_max: int, widths: dict, seed: int = 0,
                slot: int = 0, info: list | None = None) -> list:
    """Compression sweep with the range finder at the bonds listed in `widths`.

    Identical to :func:`oracle.qtt.compress` (left-to-right QR, then
    right-to-left cuts) except at the bonds b (1 .. n-1, bond b joins sites
    b and b+1 counted from 1) with an entry widths[b] = w: there Algorithm
    4.1 runs on the D_b x (4 D_{b+1}) unfolding with key
    bond_key(seed, slot, b); if the outside weight
    exceeds ACCEPT eps^2 |M|^2 the full SVD is used instead.  `info`, if given,
    receives (bond, used_range_finder, outside, |M|^2) per such bond.
    """
    A = [np.array(c, dtype=np.float64, copy=True) for c in cores]
    n = len(A)
    for k in range(n - 1):
        Dl, d, Dr = A[k].shape
        Qm, R = np.linalg.qr(A[k].reshape(Dl * d, Dr))
        A[k] = Qm.reshape(Dl, d, Qm.shape[1])
        A[k + 1] = np.tensordot(R, A[k + 1], axes=(1, 0))
    for k in range(n - 1, 0, -1):
        Dl, d, Dr = A[k].shape
        M = A[k].reshape(Dl, d * Dr)
        bond = k
        used = False
        if bond in widths:
            Qm, B, outside = range_finder(M, int(widths[bond]), bond_key(seed, slot, bond))
            nM = float(np.sum(M * M))
            if not outside > ACCEPT * eps * eps * nM:
                Ub, S, Vt = np.linalg.svd(B, full_matrices=False)
                r = trunc_rank_total(S, outside, eps, chi_max)
                A[k] = Vt[:r].reshape(r, d, Dr)
                A[k - 1] = np.tensordot(A[k - 1], (Qm @ Ub[:, :r]) * S[:r], axes=(2, 0))
                used = True
            if info is not None:
                info.append((bond, used, outside, nM))
        if not used:
            U, S, Vt = np.linalg.svd(M, full_matrices=False)
            r = Q.trunc_rank(S, eps, chi_max)
            A[k] = Vt[:r].reshape(r, d, Dr)
            A[k - 1] = np.tensordot(A[k - 1], U[:, :r] * S[:r], axes=(2, 0))
    return A


# ------------------------------------------------------------ features
def features(sigma: np.ndarray, bond: int, n: int) -> np.ndarray:
    """The 33 inputs of the perceptron for one bond."""
    s = np.sort(np.asarray(sigma, dtype=np.float64))[::-1]
    f = np.full(N_FEAT, -1.0)
    if s.size and s[0] > 0.0:
        v = np.log10(np.maximum(s[:32] / s[0], 1e-300))
        f[: v.size] = np.maximum(v, -16.0) / 16.0
    f[32] = bond / n
    return f


# ---------------------------------------------------------------- MLP
def unpack(p: np.ndarray):
    """Parameter vector -> (W1 (64 x 33), b1 (64), W2 (64), b2 (scalar))."""
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + N_HID * N_FEAT].reshape(N_HID, N_FEAT)
    o += N_HID * N_FEAT
    b1 = p[o:o + N_HID]
    o += N_HID
    W2 = p[o:o + N_HID]
    o += N_HID
    return W1, b1, W2, float(p[o])


def forward(p, X):
    """Outputs for the rows of X (N x 33)."""
    W1, b1, W2, b2 = unpack(p)
    Z = np.asarray(X, dtype=np.float64) @ W1.T + b1
    return np.maximum(Z, 0.0) @ W2 + b2


def loss_and_grad(p, X, y):
    """Mean squared error and its gradient (back-propagation written out)."""
    W1, b1, W2, b2 = unpack(p)
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    N = X.shape[0]
    Z = X @ W1.T + b1                  # N x 64
    A = np.maximum(Z, 0.0)
    out = A @ W2 + b2                  # N
    r = out - y
    L = float(np.mean(r * r))
    dout = 2.0 * r / N                 # dL/dout
    gW2 = A.T @ dout
    gb2 = float(dout.sum())
    dA = np.outer(dout, W2)
    dZ = dA * (Z > 0.0)
    gW1 = dZ.T @ X
    gb1 = dZ.sum(axis=0)
    return L, np.concatenate([gW1.ravel(), gb1, gW2, [gb2]])


def adam_step(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step number t >= 1); returns new (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def init_params(seed: int = 0) -> np.ndarray:
    """He-style initial weights (seeded numpy; the GPU side receives them)."""
    rng = np.random.default_rng(seed)
    W1 = rng.standard_normal((N_HID, N_FEAT)) * np.sqrt(2.0 / N_FEAT)
    W2 = rng.standard_normal(N_HID) * np.sqrt(1.0 / N_HID)
    return np.concatenate([W1.ravel(), np.zeros(N_HID), W2, [0.0]])


def predict_rank(p, f: np.ndarray, chi_max: int) -> int:
    out = float(forward(p, f[None, :])[0])
    return int(min(max(round(out * chi_max), 1), chi_max))
