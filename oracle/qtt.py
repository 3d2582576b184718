"""QTT / MPS oracle: the paper's algorithm in plain numpy FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Conventions (paper Sec. II.B, "quantics" encoding and Eq. for the MPS):
  * a velocity component on the periodic N x N grid, N = 2**n, is the array
    F[x1, x2] (x1 slow); bit k of x_i (k = 1 most significant) is x_i^k;
  * site k carries the physical index omega_k = 2 * x1^k + x2^k (dim 4);
  * an MPS is a list of n cores, core k of shape (D_{k-1}, 4, D_k),
    D_0 = D_n = 1;
  * an MPO is a list of n cores W[p, s_out, s_in, q] of shape
    (w_{k-1}, 4, 4, w_k) with the boundary vectors folded in (w_0 = w_n = 1);
    applied to a state it maps the coefficient at s_in to s_out.

Where the paper is silent or ambiguous, the docstring of the function
concerned states the reading it implements.

parity: pinned by tests/test_oracle_*.py (carry table of App. A, dense
stencils, Fourier-space projection, closed forms and invariants).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

D_PHYS = 4


td = np.tensordot   # pairwise contractions below are plain matrix products


def env_left(E, vi, K, vj):
    """E'[b,q,z] = sum E[a,p,x] vi[a,s,b] K[p,s,t,q] vj[x,t,z]."""
    t = td(E, vj, ([2], [0]))              # a p t z
    t = td(t, K, ([1, 2], [0, 2]))         # a z s q
    t = td(t, vi, ([0, 2], [0, 1]))        # z q b
    return t.transpose(2, 1, 0)


def env_right(E, vi, K, vj):
    """E'[a,p,x] = sum vi[a,s,b] K[p,s,t,q] vj[x,t,z] E[b,q,z]."""
    t = td(vj, E, ([2], [2]))              # x t b q
    t = td(t, K, ([1, 3], [2, 3]))         # x b p s
    t = td(t, vi, ([1, 3], [2, 1]))        # x p a
    return t.transpose(2, 1, 0)


def local_apply(LE, K, X, RE):
    """Y[a,s,b] = sum LE[a,p,x] K[p,s,t,q] X[x,t,z] RE[b,q,z]."""
    t = td(LE, X, ([2], [0]))              # a p t z
    t = td(t, K, ([1, 2], [0, 2]))         # a z s q
    return td(t, RE, ([1, 3], [2, 1]))     # a s b


def ovl_left(E, vi, wi):
    """E'[b,d] = sum E[a,c] vi[a,s,b] wi[c,s,d]."""
    return td(vi, td(E, wi, ([1], [0])), ([0, 1], [0, 1]))


def ovl_right(E, vi, wi):
    """E'[a,c] = sum vi[a,s,b] wi[c,s,d] E[b,d]."""
    return td(vi, td(wi, E, ([2], [1])), ([1, 2], [1, 2]))


def local_rhs(LW, wi, RW):
    """b[a,s,b] = sum LW[a,c] wi[c,s,d] RW[b,d]."""
    return td(td(LW, wi, ([1], [0])), RW, ([2], [1]))


# --------------------------------------------------------------------------
# Encoding (Sec. II.B, quantics representation)
# --------------------------------------------------------------------------
def dense_to_tensor(F: np.ndarray) -> np.ndarray:
    """Reorder F[x1, x2] into the tensor U[omega_1, ..., omega_n].

    omega_k = (x1^k x2^k)_2, site 1 holding the most significant bits
    (Sec. II.B).
    """
    N = F.shape[0]
    n = int(round(math.log2(N)))
    assert F.shape == (N, N) and 2 ** n == N
    T = F.reshape((2,) * n + (2,) * n)  # x1^1..x1^n, x2^1..x2^n
    perm = [ax for k in range(n) for ax in (k, n + k)]
    return T.transpose(perm).reshape((D_PHYS,) * n)


def tensor_to_dense(T: np.ndarray, n: int) -> np.ndarray:
    """Inverse of :func:`dense_to_tensor`."""
    T = np.asarray(T).reshape((2, 2) * n)  # x1^1, x2^1, x1^2, x2^2, ...
    perm = list(range(0, 2 * n, 2)) + list(range(1, 2 * n, 2))
    return T.transpose(perm).reshape(2 ** n, 2 ** n)


def trunc_rank(s: np.ndarray, eps: float, chi_max: int) -> int:
    """Rank kept at one bond (Sec. III.E, Eq. for epsilon).

    The paper defines epsilon for a whole state only; here it is applied
    per bond, relative to that bond's own weight: the smallest r >= 1 whose
    discarded weight sum_{j>r} s_j^2 is at most eps^2 * sum_j s_j^2, then
    capped at chi_max.  s is sorted descending.  An all-zero spectrum keeps
    rank 1.
    """
    s2 = np.asarray(s, dtype=np.float64) ** 2
    m = s2.shape[0]
    total = float(s2.sum())
    if total == 0.0 or m == 0:
        return 1
    # tail[j] = sum_{i >= j} s2[i], summed from the small end
    tail = np.zeros(m + 1)
    for j in range(m - 1, -1, -1):
        tail[j] = tail[j + 1] + s2[j]
    thr = eps * eps * total
    r = m
    for cand in range(1, m + 1):
        if tail[cand] <= thr:
            r = cand
            break
    return max(1, min(r, chi_max))


def from_dense(F: np.ndarray, eps: float, chi_max: int) -> list:
    """TT-SVD of a dense field into a QTT (Sec. II.B; truncation of Sec. III.E).

    Right to left: at each bond the unfolding (sites 1..k) x (site k+1 and
    the carried rank) is split by an SVD, the rank is chosen by
    :func:`trunc_rank`, V^T becomes core k+1 and U S carries on, so the
    result has its centre at site 1 like every compression.
    """
    n = int(round(math.log2(F.shape[0])))
    M = dense_to_tensor(np.asarray(F, dtype=np.float64)).reshape(-1)
    cores = [None] * n
    r_right = 1
    for k in range(n - 1, 0, -1):
        M = M.reshape(D_PHYS ** k, D_PHYS * r_right)
        U, S, Vt = np.linalg.svd(M, full_matrices=False)
        r = trunc_rank(S, eps, chi_max)
        cores[k] = Vt[:r].reshape(r, D_PHYS, r_right).copy()
        M = U[:, :r] * S[:r]
        r_right = r
    cores[0] = M.reshape(1, D_PHYS, r_right).copy()
    return cores


def to_dense(cores: list) -> np.ndarray:
    """Contract the cores left to right and undo the interleaving."""
    n = len(cores)
    T = np.ones((1, 1))
    for A in cores:
        T = np.tensordot(T, A, axes=(1, 0)).reshape(-1, A.shape[2])
    return tensor_to_dense(T.reshape(-1), n)


def bond_dims(cores: list) -> list:
    return [1] + [int(A.shape[2]) for A in cores]


def inner(A: list, B: list) -> float:
    """<a|b> by transfer matrices."""
    E = np.ones((1, 1))
    for a, b in zip(A, B):
        E = ovl_left(E, a, b)
    return float(E[0, 0])


def norm2(A: list) -> float:
    return inner(A, A)


# --------------------------------------------------------------------------
# MPOs (Sec. II.B and App. A, Table "diff_mpo")
# --------------------------------------------------------------------------
def carry_core(axis: int) -> np.ndarray:
    """Central rank-4 tensor C[alpha_m, omega_m, omega'_m, alpha_{m+1}].

    App. A: alpha_{m+1} is the request coming from the less significant
    bits (0: keep, 1: add 1, 2: subtract 1) applied to the x-bit (axis 1)
    or, "using the same logic" (Sec. II.B), to the y-bit (axis 2) of
    omega_m; alpha_m is the carry / borrow passed to the more significant
    site.  The table is read with omega_m as the output index and omega'_m
    as the input index, so that the assembled operator computes
    (U(x+1) - U(x-1)) / (2 dx); tests pin this against the dense stencil.
    """
    assert axis in (1, 2)
    C = np.zeros((3, D_PHYS, D_PHYS, 3))
    for q in range(3):
        for s_out in range(D_PHYS):
            x, y = s_out >> 1, s_out & 1
            bit = x if axis == 1 else y
            if q == 0:
                nb, p = bit, 0
            elif q == 1:
                nb = bit + 1
                p = 1 if nb == 2 else 0
                nb %= 2
            else:
                nb = bit - 1
                p = 2 if nb == -1 else 0
                nb %= 2
            s_in = (nb << 1 | y) if axis == 1 else (x << 1 | nb)
            C[p, s_out, s_in, q] = 1.0
    return C


def mpo_diff(n: int, axis: int, dx: float) -> list:
    """Central-difference MPO D_axis (App. A).

    L = (1, 1, 1) on the most significant side drops the final carry
    (periodic wrap), R = (0, 1, -1) / (2 dx) on the least significant side
    starts the +1 / -1 branches.  The grid is periodic, so the spacing is
    dx = L_domain / N (the paper's 1/(N-1) would not close the period).
    """
    C = carry_core(axis)
    L = np.ones(3)
    R = np.array([0.0, 1.0, -1.0]) / (2.0 * dx)
    W = [C.copy() for _ in range(n)]
    W[0] = np.einsum("p,pstq->stq", L, W[0])[None]
    W[-1] = np.einsum("pstq,q->pst", W[-1], R)[..., None]
    return W


def central_weights(order: int) -> np.ndarray:
    """Weights c_1..c_m (m = order / 2) of the central difference of the
    given even order, D U(x) = sum_k c_k (U(x + k dx) - U(x - k dx)) / dx
    (Sec. II.B: finite-difference operators of any order; App. D uses an
    8th-order stencil).  From the Taylor expansion, the difference
    U(x + k dx) - U(x - k dx) holds only odd derivatives, so D U = U' + O(dx^order)
    requires sum_k c_k k = 1/2 and sum_k c_k k^j = 0 for odd j = 3..order-1:
    m linear equations, solved here."""
    assert order >= 2 and order % 2 == 0
    m = order // 2
    k = np.arange(1, m + 1, dtype=np.float64)
    A = np.array([k ** (2 * i + 1) for i in range(m)])
    rhs = np.zeros(m)
    rhs[0] = 0.5
    return np.linalg.solve(A, rhs)


def mpo_shift(n: int, axis: int, a: int) -> list:
    """S^a along one axis, (S^a U)(x) = U(x + a e_axis) on the periodic grid,
    as the binary addition of the integer a to that axis' bits (the carry
    logic of App. A, Table "diff_mpo", for any constant).  Reading the bits
    from the least significant site upwards, the bond carries the value p
    still to be added to the more significant part: at a site with output
    bit b and incoming p, the input bit is (b + p) mod 2 and the outgoing
    value floor((b + p) / 2).  The value left over at the most significant
    site is a multiple of N and is dropped (periodic wrap).  Bond states are
    the values reachable from a at each bond."""
    states = [None] * (n + 1)
    states[n] = [a]
    for k in range(n - 1, -1, -1):
        nxt = sorted({(b + p) // 2 for p in states[k + 1] for b in (0, 1)})
        states[k] = nxt
    W = []
    for k in range(n):
        left, right = states[k], states[k + 1]
        w = np.zeros((len(left), D_PHYS, D_PHYS, len(right)))
        for qi, p in enumerate(right):
            for s_out in range(D_PHYS):
                x, y = s_out >> 1, s_out & 1
                b = x if axis == 1 else y
                nb, carry = (b + p) % 2, (b + p) // 2
                s_in = (nb << 1 | y) if axis == 1 else (x << 1 | nb)
                w[left.index(carry), s_out, s_in, qi] = 1.0
        W.append(w)
    W[0] = W[0].sum(axis=0)[None]   # drop the final carry
    return W


def mpo_scale(W: list, c: float) -> list:
    out = [w.copy() for w in W]
    out[0] = out[0] * c
    return out


def mpo_diff_order(n: int, axis: int, dx: float, order: int) -> list:
    """Central difference of the given even order along one axis,
    sum_k c_k (S^k - S^-k) / dx with the weights of central_weights, as a
    compressed sum of shift MPOs.  Order 2 is the paper's D (App. A)."""
    c = central_weights(order)
    W = None
    for k in range(1, len(c) + 1):
        for sign in (1, -1):
            t = mpo_scale(mpo_shift(n, axis, sign * k), sign * c[k - 1] / dx)
            W = t if W is None else mpo_sum(W, t)
    return mpo_compress(W)


def mpo_transpose(W: list) -> list:
    return [w.transpose(0, 2, 1, 3).copy() for w in W]


def mpo_product(A: list, B: list) -> list:
    """The MPO of A.B (B acts first): sum over the shared physical index."""
    out = []
    for a, b in zip(A, B):
        t = np.einsum("pxtq,rtys->prxyqs", a, b)
        pa, pb, _, _, qa, qb = t.shape
        out.append(t.reshape(pa * pb, D_PHYS, D_PHYS, qa * qb))
    return out


def mpo_sum(A: list, B: list) -> list:
    """Block-diagonal sum of two MPOs (bonds add)."""
    n = len(A)
    out = []
    for k, (a, b) in enumerate(zip(A, B)):
        if n == 1:
            out.append(a + b)
        elif k == 0:
            out.append(np.concatenate([a, b], axis=3))
        elif k == n - 1:
            out.append(np.concatenate([a, b], axis=0))
        else:
            pa, _, _, qa = a.shape
            pb, _, _, qb = b.shape
            t = np.zeros((pa + pb, D_PHYS, D_PHYS, qa + qb))
            t[:pa, :, :, :qa] = a
            t[pa:, :, :, qa:] = b
            out.append(t)
    return out


def mpo_compress(W: list, rel_tol: float = 1e-13) -> list:
    """Exact (up to rounding) bond reduction of an MPO by the MPS sweep.

    The MPO is read as an MPS with physical dimension 16; singular values
    below rel_tol times the largest at that bond are dropped.
    """
    A = [w.reshape(w.shape[0], D_PHYS * D_PHYS, w.shape[3]) for w in W]
    n = len(A)
    for k in range(n - 1):
        Dl, d, Dr = A[k].shape
        Q, R = np.linalg.qr(A[k].reshape(Dl * d, Dr))
        A[k] = Q.reshape(Dl, d, -1)
        A[k + 1] = np.tensordot(R, A[k + 1], axes=(1, 0))
    for k in range(n - 1, 0, -1):
        Dl, d, Dr = A[k].shape
        U, S, Vt = np.linalg.svd(A[k].reshape(Dl, d * Dr), full_matrices=False)
        r = max(1, int(np.sum(S > rel_tol * S[0]))) if S[0] > 0 else 1
        A[k] = Vt[:r].reshape(r, d, Dr)
        A[k - 1] = np.tensordot(A[k - 1], U[:, :r] * S[:r], axes=(2, 0))
    return [a.reshape(a.shape[0], D_PHYS, D_PHYS, a.shape[2]) for a in A]


def tensor_index(x1: int, x2: int, n: int) -> int:
    """Flat omega-ordered index of grid point (x1, x2)."""
    idx = 0
    for k in range(n):
        b1 = (x1 >> (n - 1 - k)) & 1
        b2 = (x2 >> (n - 1 - k)) & 1
        idx = idx * D_PHYS + (2 * b1 + b2)
    return idx


def mpo_to_dense(W: list) -> np.ndarray:
    """Dense N^2 x N^2 matrix of an MPO in grid order (x1, x2): brute force,
    small n only."""
    n = len(W)
    T = np.ones((1, 1, 1))  # (out, in, bond)
    for w in W:
        T = np.einsum("abp,pxyq->axbyq", T, w)
        o, _, i, _, q = T.shape
        T = T.reshape(o * D_PHYS, i * D_PHYS, q)
    M = T[:, :, 0]
    N = 2 ** n
    perm = np.array([tensor_index(x1, x2, n) for x1 in range(N) for x2 in range(N)])
    return M[np.ix_(perm, perm)]


@dataclasses.dataclass
class Operators:
    """The MPOs one time step needs, built once (App. A, App. B)."""
    n: int
    dx: float
    D: list            # [D_1, D_2]
    lap: list          # D_1 D_1 + D_2 D_2, the literal square of the central difference
    K: dict            # (i, j) -> D_i^T D_j, the blocks of the projection system
    order: int = 2     # order of the central differences


def build_operators(n: int, dx: float, order: int = 2) -> Operators:
    """D_1, D_2 (App. A for order 2; the higher even orders of Sec. II.B by
    mpo_diff_order), the Laplacian D_1 D_1 + D_2 D_2 and the projection
    blocks D_i^T D_j."""
    if order == 2:
        D1 = mpo_diff(n, 1, dx)
        D2 = mpo_diff(n, 2, dx)
    else:
        D1 = mpo_diff_order(n, 1, dx, order)
        D2 = mpo_diff_order(n, 2, dx, order)
    lap = mpo_compress(mpo_sum(mpo_compress(mpo_product(D1, D1)),
                               mpo_compress(mpo_product(D2, D2))))
    D = [D1, D2]
    K = {}
    for i in range(2):
        for j in range(2):
            K[(i, j)] = mpo_compress(mpo_product(mpo_transpose(D[i]), D[j]))
    return Operators(n=n, dx=dx, D=D, lap=lap, K=K, order=order)


# --------------------------------------------------------------------------
# MPS algebra (Sec. II.B-II.C)
# --------------------------------------------------------------------------
def compress(cores: list, eps: float, chi_max: int) -> list:
    """Compression sweep to (eps, chi_max) (Sec. II.C, "repeated SVDs").

    Left to right: QR of the (D_{k-1}*4) x D_k unfolding, R pushed into the
    next core.  Right to left: SVD of the D_{k-1} x (4*D_k) unfolding, rank
    by :func:`trunc_rank`, V^T kept as the core and U*S pushed into the
    previous core.  The result has its centre at site 1 (sites 2..n are
    right isometries).
    """
    A = [np.array(c, dtype=np.float64, copy=True) for c in cores]
    n = len(A)
    for k in range(n - 1):
        Dl, d, Dr = A[k].shape
        Q, R = np.linalg.qr(A[k].reshape(Dl * d, Dr))
        A[k] = Q.reshape(Dl, d, Q.shape[1])
        A[k + 1] = np.tensordot(R, A[k + 1], axes=(1, 0))
    for k in range(n - 1, 0, -1):
        Dl, d, Dr = A[k].shape
        U, S, Vt = np.linalg.svd(A[k].reshape(Dl, d * Dr), full_matrices=False)
        r = trunc_rank(S, eps, chi_max)
        A[k] = Vt[:r].reshape(r, d, Dr)
        A[k - 1] = np.tensordot(A[k - 1], U[:, :r] * S[:r], axes=(2, 0))
    return A


def apply_mpo_exact(W: list, A: list) -> list:
    """MPO x MPS site by site: out[(a,p), s', (b,q)] = sum_s W[p,s',s,q] A[a,s,b].

    Bonds multiply by the MPO bond (Sec. II.B: MPOs act by contracting the
    physical indices).
    """
    out = []
    for w, a in zip(W, A):
        t = np.einsum("pxsq,asb->apxbq", w, a)
        da, pw, _, db, qw = t.shape
        out.append(t.reshape(da * pw, D_PHYS, db * qw))
    return out


def apply_mpo(W, A, eps, chi_max):
    return compress(apply_mpo_exact(W, A), eps, chi_max)


def add_exact(coefs, terms) -> list:
    """Block-diagonal MPS sum sum_t c_t |t> (Sec. II.C "addition step").

    The coefficients scale the first core; bonds add.
    """
    n = len(terms[0])
    out = []
    for k in range(n):
        blocks = [t[k] for t in terms]
        if k == 0:
            blocks = [c * b for c, b in zip(coefs, blocks)]
        if n == 1:
            out.append(sum(blocks))
        elif k == 0:
            out.append(np.concatenate(blocks, axis=2))
        elif k == n - 1:
            out.append(np.concatenate(blocks, axis=0))
        else:
            Dl = sum(b.shape[0] for b in blocks)
            Dr = sum(b.shape[2] for b in blocks)
            t = np.zeros((Dl, D_PHYS, Dr))
            i0 = j0 = 0
            for b in blocks:
                t[i0:i0 + b.shape[0], :, j0:j0 + b.shape[2]] = b
                i0 += b.shape[0]
                j0 += b.shape[2]
            out.append(t)
    return out


def add(coefs, terms, eps, chi_max):
    return compress(add_exact(coefs, terms), eps, chi_max)


def hadamard_exact(A, B) -> list:
    """Element-wise product |a> (.) |b> with bond Da*Db (Sec. II.B, copy
    tensors delta_{omega omega omega})."""
    out = []
    for a, b in zip(A, B):
        t = np.einsum("asc,bsd->abscd", a, b)
        da, db, _, dc, dd = t.shape
        out.append(t.reshape(da * db, D_PHYS, dc * dd))
    return out


def hadamard(A, B, eps, chi_max) -> list:
    """Hadamard product by zip-up, then a compression sweep (Sec. II.B).

    The chi^2 product bond is never formed.  A carry R[r, a, b] runs left
    to right; at site k the contraction
    T[r, s, a', b'] = sum_{a,b} R[r,a,b] A_k[a,s,a'] B_k[b,s,b'] is split
    by an SVD of its (r*4) x (a'*b') unfolding, keeping
    min(4r, a'b', chi_max) directions (a cap only: the eps decision is left
    to the final sweep, whose environments are orthonormal), U becoming the
    core and S V^T the new carry.  A full compress(eps, chi_max) follows.
    """
    n = len(A)
    R = np.ones((1, 1, 1))
    C = []
    for k in range(n):
        T = np.stack([td(td(R, A[k][:, s, :], ([1], [0])), B[k][:, s, :], ([1], [0]))
                      for s in range(D_PHYS)], axis=1)      # r s a' b'
        r = T.shape[0]
        if k == n - 1:
            C.append(T.reshape(r, D_PHYS, 1))
            break
        dc, dd = T.shape[2], T.shape[3]
        M = T.reshape(r * D_PHYS, dc * dd)
        U, S, Vt = np.linalg.svd(M, full_matrices=False)
        rk = max(1, min(S.shape[0], chi_max))
        C.append(U[:, :rk].reshape(r, D_PHYS, rk))
        R = (S[:rk, None] * Vt[:rk]).reshape(rk, dc, dd)
    return compress(C, eps, chi_max)


# --------------------------------------------------------------------------
# Variational projection (App. B, Eqs. "first", "second", "big_LS")
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Params:
    """Solver parameters; defaults are the paper's (Sec. II.C, App. B)."""
    eps: float = 1e-8
    chi_max: int = 64
    mu: float = 2.5e5
    cg_tol: float = 1e-5
    cg_maxit: int = 100
    sweep_tol: float = 1e-5
    max_sweeps: int = 20
    projection: str = "penalty"   # or "spectral": project_spectral in every stage


def right_canonicalize(A: list) -> list:
    """Right-to-left QR sweep: sites 2..n become right isometries."""
    A = [a.copy() for a in A]
    for k in range(len(A) - 1, 0, -1):
        Dl, d, Dr = A[k].shape
        Q, R = np.linalg.qr(A[k].reshape(Dl, d * Dr).T)
        A[k] = Q.T.reshape(Q.shape[1], d, Dr)
        A[k - 1] = np.tensordot(A[k - 1], R.T, axes=(2, 0))
    return A


@dataclasses.dataclass
class ProjectInfo:
    sweeps: int = 0
    cg_iters: int = 0
    converged: bool = False


def project(w: list, h: float, params: Params, ops: Operators):
    """Minimise mu |D1 v1 + D2 v2|^2 + |v - w|^2 / h^2 over MPS pairs v.

    This is the cost Theta of App. B with w_i = a_i - h B_i formed
    explicitly as an MPS and the cost multiplied by h^2; its stationarity
    condition is the coupled system "big_LS",
    (1 + mu h^2 sum_j D_i^T D_j) C = <basis|w> (Eqs. "first"/"second"
    with D^T = -D).  DMRG-like single-site sweeps (Sec. II.C): both
    components share the centre site d; the local system is solved by CG
    with the operator kept factored (Sec. II.D); the centre moves by QR
    (QR and SVD give the same state when no bond is truncated).  One
    sweep = sites 1..n-1 left to right, then n..2 right to left, so the
    centre returns to site 1; sweeps stop when the relative change of
    sum_i <v_i|v_i> over one sweep is <= sweep_tol.  Initial guess: w
    itself, brought to right-canonical form (the paper starts from the
    previous time step; w is already rank-adapted by its compression).
    """
    n = ops.n
    c = params.mu * h * h
    V = [right_canonicalize(w[0]), right_canonicalize(w[1])]
    W = [w[0], w[1]]
    blocks = [(i, j) for i in range(2) for j in range(2)]

    one3 = np.ones((1, 1, 1))
    one2 = np.ones((1, 1))
    LE = {b: [None] * (n + 1) for b in blocks}
    RE = {b: [None] * (n + 1) for b in blocks}
    LW = [[None] * (n + 1) for _ in range(2)]
    RW = [[None] * (n + 1) for _ in range(2)]
    for b in blocks:
        LE[b][0] = one3
        RE[b][n] = one3
    for i in range(2):
        LW[i][0] = one2
        RW[i][n] = one2

    def build_right(k):
        """Environments of sites k..n-1 (0-based), stored at index k."""
        for (i, j) in blocks:
            RE[(i, j)][k] = env_right(RE[(i, j)][k + 1], V[i][k], ops.K[(i, j)][k], V[j][k])
        for i in range(2):
            RW[i][k] = ovl_right(RW[i][k + 1], V[i][k], W[i][k])

    def build_left(k):
        """Environments of sites 0..k-1 (0-based), stored at index k."""
        for (i, j) in blocks:
            LE[(i, j)][k] = env_left(LE[(i, j)][k - 1], V[i][k - 1], ops.K[(i, j)][k - 1],
                                     V[j][k - 1])
        for i in range(2):
            LW[i][k] = ovl_left(LW[i][k - 1], V[i][k - 1], W[i][k - 1])

    for k in range(n - 1, 0, -1):
        build_right(k)

    info = ProjectInfo()

    def matvec(d, X):
        Y = [X[0].copy(), X[1].copy()]
        for (i, j) in blocks:
            Y[i] += c * local_apply(LE[(i, j)][d], ops.K[(i, j)][d], X[j], RE[(i, j)][d + 1])
        return Y

    def solve(d):
        rhs = [local_rhs(LW[i][d], W[i][d], RW[i][d + 1]) for i in range(2)]
        x = [V[0][d].copy(), V[1][d].copy()]
        its = conjugate_gradient(lambda X: matvec(d, X), rhs, x, params.cg_tol, params.cg_maxit)
        info.cg_iters += its
        V[0][d], V[1][d] = x

    def norm_total():
        return float(sum(np.sum(V[i][0] ** 2) for i in range(2)))

    n_prev = norm_total()
    for sweep in range(params.max_sweeps):
        for d in range(0, n - 1):
            solve(d)
            for i in range(2):
                Dl, dd, Dr = V[i][d].shape
                Q, R = np.linalg.qr(V[i][d].reshape(Dl * dd, Dr))
                V[i][d] = Q.reshape(Dl, dd, Q.shape[1])
                V[i][d + 1] = np.tensordot(R, V[i][d + 1], axes=(1, 0))
            build_left(d + 1)
        for d in range(n - 1, 0, -1):
            solve(d)
            for i in range(2):
                Dl, dd, Dr = V[i][d].shape
                Q, R = np.linalg.qr(V[i][d].reshape(Dl, dd * Dr).T)
                V[i][d] = Q.T.reshape(Q.shape[1], dd, Dr)
                V[i][d - 1] = np.tensordot(V[i][d - 1], R.T, axes=(2, 0))
            build_right(d)
        info.sweeps = sweep + 1
        n_new = norm_total()
        if n_new == 0.0 or abs(n_new - n_prev) <= params.sweep_tol * n_new:
            info.converged = True
            break
        n_prev = n_new
    return V, info


def project_spectral(w: list, params: Params, ops: Operators):
    """The exact discrete projection of w onto divergence-free fields, the
    alternative to the penalty that the paper's outlook (Sec. IV) points to
    for periodic boundaries: both components are read out densely, the
    divergence is removed exactly per Fourier mode (oracle.dense.project_exact,
    the mu -> infinity limit of the penalty solve), and each component is
    encoded again by TT-SVD to (eps, chi_max) (`from_dense`)."""
    from oracle import dense as Dn
    v = Dn.project_exact([to_dense(w[0]), to_dense(w[1])], ops.dx, ops.order)
    return [from_dense(v[i], params.eps, params.chi_max) for i in range(2)], ProjectInfo()


def project_stage(w: list, h: float, params: Params, ops: Operators):
    """The projection of one Euler minimisation: the penalty solve
    (`project`, the paper's) or, with params.projection == "spectral",
    `project_spectral`."""
    if params.projection == "spectral":
        return project_spectral(w, params, ops)
    return project(w, h, params, ops)


def hadamard_mpo(Y: list) -> list:
    """The MPO H_Y of the element-wise product with the MPS Y:
    H_Y[c, s, t, c'] = Y[c, s, c'] delta(s, t), so that H_Y X = Y (.) X
    (Sec. II.B: the Hadamard product as a "nonlinear MPO")."""
    eye = np.eye(D_PHYS)
    return [np.einsum("asb,st->astb", y, eye) for y in Y]


def implicit_terms(u, b, h: float, nu: float, ops: Operators, a_scale: float = 0.25):
    """The right-hand side a u_i - h B_i(b) of one penalised Euler
    minimisation as a sum of networks that are never contracted into an MPS
    (the paper's form of the step, Sec. II.C and App. B, Eq. for B_i inside
    the cost Theta): for component i a list of (coef, P, X) with P an MPO
    (None: the identity) applied to the MPS X,
      a_scale u_i                              (coef a_scale, P = I, X = u_i)
      - h/2 b_j (.) D_j b_i = -h/2 (H_{b_j} D_j) b_i      (j = 1, 2)
      - h/2 D_j (b_j (.) b_i) = -h/2 (D_j H_{b_j}) b_i    (j = 1, 2)
      + h nu (D_1 D_1 + D_2 D_2) b_i           (the literal squares, reading 3).
    """
    terms = [[], []]
    for i in range(2):
        terms[i].append((a_scale, None, u[i]))
        for j in range(2):
            Hj = hadamard_mpo(b[j])
            terms[i].append((-0.5 * h, mpo_product(Hj, ops.D[j]), b[i]))
            terms[i].append((-0.5 * h, mpo_product(ops.D[j], Hj), b[i]))
        terms[i].append((h * nu, ops.lap, b[i]))
    return terms


def project_implicit(terms, guess, h: float, params: Params, ops: Operators):
    """The projection of `project` with the right-hand side given as the
    networks of `implicit_terms` instead of an MPS w (the paper's form,
    Sec. II.C: the nonlinear MPOs are contracted with the velocity states
    inside the local problem).  The local right-hand side of component i at
    the centre d is sum_t coef_t <L_t| P_t X_t |R_t>, with environments of
    V_i against each term (overlaps for P = I, MPO sandwiches otherwise),
    updated as the centre moves.  Initial guess `guess` (the paper: the
    previous time step), brought to right-canonical form; its bonds are kept.
    Same sweeps, CG and stopping rules as `project`."""
    n = ops.n
    c = params.mu * h * h
    V = [right_canonicalize(guess[0]), right_canonicalize(guess[1])]
    blocks = [(i, j) for i in range(2) for j in range(2)]
    one3 = np.ones((1, 1, 1))
    one2 = np.ones((1, 1))
    LE = {bk: [None] * (n + 1) for bk in blocks}
    RE = {bk: [None] * (n + 1) for bk in blocks}
    nt = [len(terms[i]) for i in range(2)]
    TL = [[[None] * (n + 1) for _ in range(nt[i])] for i in range(2)]
    TR = [[[None] * (n + 1) for _ in range(nt[i])] for i in range(2)]
    for bk in blocks:
        LE[bk][0] = one3
        RE[bk][n] = one3
    for i in range(2):
        for t, (_, P, _) in enumerate(terms[i]):
            TL[i][t][0] = one2 if P is None else one3
            TR[i][t][n] = one2 if P is None else one3

    def build_right(k):
        for (i, j) in blocks:
            RE[(i, j)][k] = env_right(RE[(i, j)][k + 1], V[i][k], ops.K[(i, j)][k], V[j][k])
        for i in range(2):
            for t, (_, P, X) in enumerate(terms[i]):
                TR[i][t][k] = (ovl_right(TR[i][t][k + 1], V[i][k], X[k]) if P is None else
                               env_right(TR[i][t][k + 1], V[i][k], P[k], X[k]))

    def build_left(k):
        for (i, j) in blocks:
            LE[(i, j)][k] = env_left(LE[(i, j)][k - 1], V[i][k - 1], ops.K[(i, j)][k - 1],
                                     V[j][k - 1])
        for i in range(2):
            for t, (_, P, X) in enumerate(terms[i]):
                TL[i][t][k] = (ovl_left(TL[i][t][k - 1], V[i][k - 1], X[k - 1]) if P is None else
                               env_left(TL[i][t][k - 1], V[i][k - 1], P[k - 1], X[k - 1]))

    for k in range(n - 1, 0, -1):
        build_right(k)

    info = ProjectInfo()

    def matvec(d, Xv):
        Y = [Xv[0].copy(), Xv[1].copy()]
        for (i, j) in blocks:
            Y[i] += c * local_apply(LE[(i, j)][d], ops.K[(i, j)][d], Xv[j], RE[(i, j)][d + 1])
        return Y

    def rhs_at(d, i):
        acc = None
        for t, (coef, P, X) in enumerate(terms[i]):
            r = (local_rhs(TL[i][t][d], X[d], TR[i][t][d + 1]) if P is None else
                 local_apply(TL[i][t][d], P[d], X[d], TR[i][t][d + 1]))
            acc = coef * r if acc is None else acc + coef * r
        return acc

    def solve(d):
        rhs = [rhs_at(d, i) for i in range(2)]
        x = [V[0][d].copy(), V[1][d].copy()]
        its = conjugate_gradient(lambda X: matvec(d, X), rhs, x, params.cg_tol, params.cg_maxit)
        info.cg_iters += its
        V[0][d], V[1][d] = x

    def norm_total():
        return float(sum(np.sum(V[i][0] ** 2) for i in range(2)))

    n_prev = norm_total()
    for sweep in range(params.max_sweeps):
        for d in range(0, n - 1):
            solve(d)
            for i in range(2):
                Dl, dd, Dr = V[i][d].shape
                Q, R = np.linalg.qr(V[i][d].reshape(Dl * dd, Dr))
                V[i][d] = Q.reshape(Dl, dd, Q.shape[1])
                V[i][d + 1] = np.tensordot(R, V[i][d + 1], axes=(1, 0))
            build_left(d + 1)
        for d in range(n - 1, 0, -1):
            solve(d)
            for i in range(2):
                Dl, dd, Dr = V[i][d].shape
                Q, R = np.linalg.qr(V[i][d].reshape(Dl, dd * Dr).T)
                V[i][d] = Q.T.reshape(Q.shape[1], dd, Dr)
                V[i][d - 1] = np.tensordot(V[i][d - 1], R.T, axes=(2, 0))
            build_right(d)
        info.sweeps = sweep + 1
        n_new = norm_total()
        if n_new == 0.0 or abs(n_new - n_prev) <= params.sweep_tol * n_new:
            info.converged = True
            break
        n_prev = n_new
    return V, info


def conjugate_gradient(matvec, b, x, tol, maxit) -> int:
    """Plain CG on a list-of-arrays vector, in place on x (App. B).

    Stops when |r| <= tol * |b| (relative residual) or after maxit
    iterations; returns the iteration count.
    """
    def dot(u, v):
        return float(sum(np.vdot(a, b_) for a, b_ in zip(u, v)))

    bnorm = math.sqrt(dot(b, b))
    if bnorm == 0.0:
        for a in x:
            a[...] = 0.0
        return 0
    Ax = matvec(x)
    r = [bi - ai for bi, ai in zip(b, Ax)]
    p = [ri.copy() for ri in r]
    rs = dot(r, r)
    it = 0
    while it < maxit and math.sqrt(rs) > tol * bnorm:
        Ap = matvec(p)
        alpha = rs / dot(p, Ap)
        for xi, pi in zip(x, p):
            xi += alpha * pi
        for ri, api in zip(r, Ap):
            ri -= alpha * api
        rs_new = dot(r, r)
        beta = rs_new / rs
        p = [ri + beta * pi for ri, pi in zip(r, p)]
        rs = rs_new
        it += 1
    return it


# --------------------------------------------------------------------------
# Right-hand side and RK4 (App. B, Eq. for B_i, Table RK4, Eqs. U1-U4)
# --------------------------------------------------------------------------
def stage_w(u, b, h, nu, params: Params, ops: Operators, a_scale: float = 0.25):
    """w_i = a_scale u_i - h B_i(b) (a_scale = 1/4 for the RK4 stages, 1 for
    the Euler and RK2 minimisations) with the skew-symmetric convection term
    B_i = sum_j 1/2 (b_j (.) D_j b_i + D_j (b_j (.) b_i)) - nu D_j^2 b_i
    (App. B, Eq. for B_i).  Every intermediate is compressed to
    (eps, chi_max); the sums are taken pairwise in the order below (the
    paper fixes none): c_a = P_0 + P_1, c_b = DQ_0 + DQ_1, conv =
    (c_a + c_b) / 2, e = a_scale u + h nu Lap b, w = e - h conv, i.e.
    w = a_scale u - h (conv - nu Lap b) with the viscous term folded into e.
    """
    eps, chi = params.eps, params.chi_max
    Db = {(j, i): apply_mpo(ops.D[j], b[i], eps, chi) for i in range(2) for j in range(2)}
    P = {(j, i): hadamard(b[j], Db[(j, i)], eps, chi) for i in range(2) for j in range(2)}
    Q = {}
    for j in range(2):
        for i in range(j, 2):
            Q[(j, i)] = hadamard(b[j], b[i], eps, chi)
    Q[(1, 0)] = Q[(0, 1)]
    DQ = {(j, i): apply_mpo(ops.D[j], Q[(j, i)], eps, chi) for i in range(2) for j in range(2)}
    Lb = [apply_mpo(ops.lap, b[i], eps, chi) for i in range(2)]
    w = []
    for i in range(2):
        ca = add([1.0, 1.0], [P[(0, i)], P[(1, i)]], eps, chi)
        cb = add([1.0, 1.0], [DQ[(0, i)], DQ[(1, i)]], eps, chi)
        e = add([a_scale, h * nu], [u[i], Lb[i]], eps, chi)
        conv = add([0.5, 0.5], [ca, cb], eps, chi)
        w.append(add([1.0, -h], [e, conv], eps, chi))
    return w


RK4_H = (1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0)        # h_s / dt, Eqs. U1-U4
RK4_B = (None, (3.0, 0.25), (1.5, 0.625), (3.0, 0.25))      # Table RK4


def rk4_step(u, dt: float, nu: float, params: Params, ops: Operators, stats=None):
    """One RK4 step as four penalised Euler minimisations (App. B, Eq.
    "4euler", Table RK4, Eqs. U1-U4); u^{s+1} = U1 + U2 + U3 + U4, summed
    left to right with a compression after each addition."""
    eps, chi = params.eps, params.chi_max
    U = []
    b = u
    for s in range(4):
        if s > 0:
            c1, c2 = RK4_B[s]
            b = [add([c1, c2], [U[s - 1][i], u[i]], eps, chi) for i in range(2)]
        h = RK4_H[s] * dt
        w = stage_w(u, b, h, nu, params, ops)
        v, info = project_stage(w, h, params, ops)
        if stats is not None:
            stats.append(info)
        U.append(v)
    out = []
    for i in range(2):
        acc = add([1.0, 1.0], [U[0][i], U[1][i]], eps, chi)
        acc = add([1.0, 1.0], [acc, U[2][i]], eps, chi)
        acc = add([1.0, 1.0], [acc, U[3][i]], eps, chi)
        out.append(acc)
    return out


def scaled(A: list, c: float) -> list:
    out = [a.copy() for a in A]
    out[0] = out[0] * c
    return out


def rk4_step_implicit(u, dt: float, nu: float, params: Params, ops: Operators, stats=None):
    """One RK4 step in the paper's form (Sec. II.C, App. B): the four
    penalised Euler minimisations of `rk4_step` (Table RK4, Eqs. U1-U4) with
    B never formed as an MPS -- each stage's right-hand side a u - h B(b)
    enters its projection as the networks of `implicit_terms`.  Initial
    guess of every stage: the previous time step, a u (a = 1/4), so each
    U_s keeps the bonds of u.  u^{s+1} = ((U1 + U2) + U3) + U4 as in
    `rk4_step`.  Identical to `rk4_step` when nothing is truncated; they
    differ by about eps otherwise."""
    eps, chi = params.eps, params.chi_max
    U = []
    b = u
    for s in range(4):
        if s > 0:
            c1, c2 = RK4_B[s]
            b = [add([c1, c2], [U[s - 1][i], u[i]], eps, chi) for i in range(2)]
        h = RK4_H[s] * dt
        terms = implicit_terms(u, b, h, nu, ops, 0.25)
        v, info = project_implicit(terms, [scaled(u[i], 0.25) for i in range(2)], h, params, ops)
        if stats is not None:
            stats.append(info)
        U.append(v)
    out = []
    for i in range(2):
        acc = add([1.0, 1.0], [U[0][i], U[1][i]], eps, chi)
        acc = add([1.0, 1.0], [acc, U[2][i]], eps, chi)
        acc = add([1.0, 1.0], [acc, U[3][i]], eps, chi)
        out.append(acc)
    return out


def euler_step(u, dt: float, nu: float, params: Params, ops: Operators):
    """One explicit Euler (RK1) step (App. B, Eq. "euler" in the cost
    function): u^{s+1} = argmin Theta(v, a = u^s, b = u^s, h = dt)."""
    w = stage_w(u, u, dt, nu, params, ops, a_scale=1.0)
    v, _ = project_stage(w, dt, params, ops)
    return v


def rk2_step(u, dt: float, nu: float, params: Params, ops: Operators):
    """One midpoint RK2 step (App. B, Eqs. "midpoint_calc", "full_calc"):
    u^{s+1/2} = argmin Theta(v, u^s, u^s, dt/2), then
    u^{s+1} = argmin Theta(v, u^s, u^{s+1/2}, dt)."""
    w = stage_w(u, u, 0.5 * dt, nu, params, ops, a_scale=1.0)
    um, _ = project_stage(w, 0.5 * dt, params, ops)
    w = stage_w(u, um, dt, nu, params, ops, a_scale=1.0)
    v, _ = project_stage(w, dt, params, ops)
    return v

