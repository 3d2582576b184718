"""Thin ctypes binding of the C ABI in include/qtt.h (argument marshalling only).

Every computation happens in libqtt_b300.so on the GPU; this module only
converts Python / torch arguments to pointers and sizes and turns status
codes into exceptions.  Importing it without the built library raises.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, byref, c_double, c_int, c_longlong, c_size_t, c_void_p

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libqtt_b300.so")

PREC_FP64 = 0
PREC_MIXED = 1
RHS_EXPLICIT = 0
RHS_IMPLICIT = 1
PROJ_PENALTY = 0
PROJ_SPECTRAL = 1
LEARNED_OFF = 0
LEARNED_LOG = 1
LEARNED_ON = 2
MLP_FEATURES = 33
MLP_HIDDEN = 64
MLP_PARAMS = MLP_HIDDEN * MLP_FEATURES + 2 * MLP_HIDDEN + 1
LEARNED_SLOTS = 512

STATUS = {0: "QTT_OK", 1: "QTT_ERR_ARG", 2: "QTT_ERR_SHAPE", 3: "QTT_ERR_ALLOC",
          4: "QTT_ERR_CUDA", 5: "QTT_ERR_NOT_CONVERGED", 6: "QTT_ERR_TIMEOUT",
          7: "QTT_ERR_NUMERIC"}
NOT_CONVERGED = 5

EXPORTS = ("qtt_create", "qtt_destroy", "qtt_set_params", "qtt_sync", "qtt_last_error",
           "qtt_from_dense", "qtt_to_dense", "qtt_mps_from_packed", "qtt_mps_to_packed",
           "qtt_mps_info", "qtt_free_mps", "qtt_mpo_get", "qtt_free_mpo", "qtt_apply_mpo",
           "qtt_add", "qtt_hadamard", "qtt_compress", "qtt_project", "qtt_rk4_step",
           "qtt_stats", "qtt_profile_begin", "qtt_profile_end", "qtt_to_dense_noalloc",
           "qtt_learned_set", "qtt_learned_next_step", "qtt_learned_log", "qtt_learned_stats",
           "qtt_rf_omega", "qtt_mlp_forward", "qtt_mlp_loss_grad", "qtt_mlp_train",
           "qtt_batch_create", "qtt_batch_destroy", "qtt_batch_context", "qtt_rk4_step_batched",
           "qtt_euler_step", "qtt_rk2_step", "qtt_inner", "qtt_graph_stats",
           "qtt_mps_upload_packed", "qtt_gemm_tf32x3", "qtt_gemm_ozaki", "qtt_tc_stats", "qtt_mpo_diff",
           "qtt_tke_spectrum", "qtt_project_spectral")


class QttError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("n", c_int), ("L", c_double), ("eps", c_double), ("chi_max", c_int),
                ("mu", c_double), ("cg_tol", c_double), ("cg_maxit", c_int),
                ("sweep_tol", c_double), ("max_sweeps", c_int), ("precision", c_int),
                ("learned_trunc", c_int), ("rf_oversample", c_int), ("rf_min_width", c_int),
                ("graphs", c_int), ("fd_order", c_int), ("rhs_form", c_int),
                ("projection", c_int)]


_lib = None


def lib():
    """Load libqtt_b300.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise ImportError(f"{_LIB_PATH} is missing: build it with "
                              "`python -m paper_2406_17823_b300.build`")
        L = ctypes.CDLL(_LIB_PATH)
        vp, ip = c_void_p, POINTER(c_int)
        sig = {
            "qtt_create": (c_int, [POINTER(vp), c_int, vp, POINTER(Params)]),
            "qtt_destroy": (c_int, [vp]),
            "qtt_set_params": (c_int, [vp, POINTER(Params)]),
            "qtt_sync": (c_int, [vp]),
            "qtt_last_error": (ctypes.c_char_p, [vp]),
            "qtt_from_dense": (c_int, [vp, vp, c_double, c_int, POINTER(vp)]),
            "qtt_to_dense": (c_int, [vp, vp, vp]),
            "qtt_mps_from_packed": (c_int, [vp, vp, c_int, ip, POINTER(vp)]),
            "qtt_mps_to_packed": (c_int, [vp, vp, vp, c_int, c_size_t, ip]),
            "qtt_mps_info": (c_int, [vp, ip, ip]),
            "qtt_free_mps": (None, [vp]),
            "qtt_mpo_get": (c_int, [vp, c_int, POINTER(vp)]),
            "qtt_mpo_diff": (c_int, [vp, c_int, c_int, c_double, POINTER(vp)]),
            "qtt_tke_spectrum": (c_int, [vp, vp, vp, c_int, POINTER(c_double)]),
            "qtt_free_mpo": (None, [vp]),
            "qtt_apply_mpo": (c_int, [vp, vp, vp, c_double, c_int, POINTER(vp)]),
            "qtt_add": (c_int, [vp, c_int, POINTER(c_double), POINTER(vp), c_double, c_int,
                                POINTER(vp)]),
            "qtt_hadamard": (c_int, [vp, vp, vp, c_double, c_int, POINTER(vp)]),
            "qtt_compress": (c_int, [vp, vp, c_double, c_int]),
            "qtt_project": (c_int, [vp, vp, vp, c_double, c_double, POINTER(vp), POINTER(vp), ip,
                                    ip]),
            "qtt_project_spectral": (c_int, [vp, vp, vp, POINTER(vp), POINTER(vp)]),
            "qtt_rk4_step": (c_int, [vp, POINTER(vp), POINTER(vp), c_double, c_double]),
            "qtt_euler_step": (c_int, [vp, POINTER(vp), POINTER(vp), c_double, c_double]),
            "qtt_inner": (c_int, [vp, vp, vp, POINTER(c_double)]),
            "qtt_rk2_step": (c_int, [vp, POINTER(vp), POINTER(vp), c_double, c_double]),
            "qtt_stats": (c_int, [vp, POINTER(c_longlong), POINTER(c_longlong),
                                  POINTER(c_longlong)]),
            "qtt_graph_stats": (c_int, [vp, POINTER(c_longlong), POINTER(c_longlong)]),
            "qtt_mps_upload_packed": (c_int, [vp, vp, vp, c_int, ip]),
            "qtt_profile_begin": (c_int, [vp]),
            "qtt_profile_end": (c_int, [vp, ctypes.c_char_p, c_size_t]),
            "qtt_to_dense_noalloc": (c_int, [vp, ip, c_int, vp, vp]),
            "qtt_tc_stats": (c_int, [vp, POINTER(c_longlong), POINTER(c_longlong)]),
            "qtt_gemm_tf32x3": (c_int, [vp, c_int, c_int, c_int, vp, c_int, c_int, vp, c_int,
                                        c_int, vp, c_int]),
            "qtt_gemm_ozaki": (c_int, [vp, c_int, c_int, c_int, vp, c_int, c_int, c_longlong, vp,
                                       c_int, c_int, c_longlong, vp, c_int, c_longlong, c_int,
                                       ctypes.c_double, ctypes.c_double]),
            "qtt_learned_set": (c_int, [vp, vp]),
            "qtt_learned_next_step": (c_int, [vp]),
            "qtt_learned_log": (c_int, [vp, vp, vp, c_int, ip]),
            "qtt_learned_stats": (c_int, [vp, POINTER(c_longlong), POINTER(c_longlong)]),
            "qtt_rf_omega": (c_int, [vp, ctypes.c_ulonglong, c_int, c_int, vp]),
            "qtt_mlp_forward": (c_int, [vp, vp, vp, c_int, vp]),
            "qtt_mlp_loss_grad": (c_int, [vp, vp, vp, vp, c_int, vp, vp]),
            "qtt_mlp_train": (c_int, [vp, vp, vp, vp, c_int, c_int, ctypes.c_float, vp]),
            "qtt_batch_create": (c_int, [POINTER(vp), c_int, c_int, POINTER(Params)]),
            "qtt_batch_destroy": (c_int, [vp]),
            "qtt_batch_context": (vp, [vp, c_int]),
            "qtt_rk4_step_batched": (c_int, [vp, POINTER(vp), POINTER(vp), POINTER(c_double),
                                             POINTER(c_double)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _torch():
    import torch
    return torch


class MPS:
    """Owning handle of a library MPS."""

    def __init__(self, ctx: "Context", handle: int):
        self.ctx = ctx
        self.h = c_void_p(handle)

    def free(self):
        if self.h and self.h.value:
            # after its context is gone (interpreter shutdown tears objects
            # down in any order) the device memory went with the context
            ctx_h = getattr(self.ctx, "h", None)
            if ctx_h is not None and ctx_h.value:
                lib().qtt_free_mps(self.h)
            self.h = c_void_p(None)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    @property
    def bonds(self):
        n = self.ctx.params.n
        b = (c_int * (n + 1))()
        self.ctx._check(lib().qtt_mps_info(self.h, None, b))
        return list(b)


class Context:
    """A library context bound to one CUDA device and the current torch stream."""

    def __init__(self, n: int, L: float = 2 * np.pi, eps: float = 1e-8, chi_max: int = 64,
                 mu: float = 2.5e5, cg_tol: float = 1e-5, cg_maxit: int = 100,
                 sweep_tol: float = 1e-5, max_sweeps: int = 20, precision: int = PREC_FP64,
                 learned_trunc: int = LEARNED_OFF, rf_oversample: int = 8,
                 rf_min_width: int = 128, graphs: int = 0, fd_order: int = 0,
                 rhs_form: int = 0, projection: int = 0, device: int = 0, stream=None):
        torch = _torch()
        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        self.params = Params(n, L, eps, chi_max, mu, cg_tol, cg_maxit, sweep_tol, max_sweeps,
                             precision, learned_trunc, rf_oversample, rf_min_width, graphs,
                             fd_order, rhs_form, projection)
        h = c_void_p()
        st = lib().qtt_create(byref(h), device, c_void_p(stream.cuda_stream), byref(self.params))
        if st != 0:
            raise QttError(st, "qtt_create failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lib().qtt_destroy(self.h)
            self.h = c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int, allow_not_converged: bool = False):
        if st == 0 or (allow_not_converged and st == NOT_CONVERGED):
            return st
        raise QttError(st, lib().qtt_last_error(self.h).decode())

    @property
    def N(self):
        return 2 ** self.params.n

    def set_params(self, **kw):
        for k, v in kw.items():
            setattr(self.params, k, v)
        self._check(lib().qtt_set_params(self.h, byref(self.params)))

    def sync(self):
        self._check(lib().qtt_sync(self.h))

    # -------------------------------------------------------------- I/O
    def from_dense(self, field, eps=None, chi_max=None) -> MPS:
        torch = _torch()
        t = torch.as_tensor(field, dtype=torch.float64, device=f"cuda:{self.device}").contiguous()
        out = c_void_p()
        self._check(lib().qtt_from_dense(self.h, c_void_p(t.data_ptr()),
                                         self.params.eps if eps is None else eps,
                                         self.params.chi_max if chi_max is None else chi_max,
                                         byref(out)))
        self._keep = t
        return MPS(self, out.value)

    def to_dense(self, mps: MPS):
        torch = _torch()
        out = torch.empty((self.N, self.N), dtype=torch.float64, device=f"cuda:{self.device}")
        self._check(lib().qtt_to_dense(self.h, mps.h, c_void_p(out.data_ptr())))
        return out

    def from_cores(self, cores) -> MPS:
        """Upload a list of numpy cores (D_{k-1}, 4, D_k) (host buffer path)."""
        bonds = [1] + [int(c.shape[2]) for c in cores]
        flat = np.ascontiguousarray(np.concatenate([np.asarray(c, np.float64).reshape(-1)
                                                    for c in cores]))
        b = (c_int * len(bonds))(*bonds)
        out = c_void_p()
        self._check(lib().qtt_mps_from_packed(self.h, c_void_p(flat.ctypes.data), 0, b,
                                              byref(out)))
        return MPS(self, out.value)

    def upload_cores(self, mps: MPS, cores):
        """Overwrite `mps` with numpy cores (host buffer path), keeping its
        capacities (each bond at most the MPS's capacity)."""
        bonds = [1] + [int(c.shape[2]) for c in cores]
        flat = np.ascontiguousarray(np.concatenate([np.asarray(c, np.float64).reshape(-1)
                                                    for c in cores]))
        b = (c_int * len(bonds))(*bonds)
        self._check(lib().qtt_mps_upload_packed(self.h, mps.h, c_void_p(flat.ctypes.data), 0, b))

    def to_cores(self, mps: MPS):
        n = self.params.n
        bonds = mps.bonds
        total = sum(bonds[k] * 4 * bonds[k + 1] for k in range(n))
        buf = np.empty(total, np.float64)
        b = (c_int * (n + 1))()
        self._check(lib().qtt_mps_to_packed(self.h, mps.h, c_void_p(buf.ctypes.data), 0, total, b))
        cores, o = [], 0
        for k in range(n):
            sz = b[k] * 4 * b[k + 1]
            cores.append(buf[o:o + sz].reshape(b[k], 4, b[k + 1]).copy())
            o += sz
        return cores

    # -------------------------------------------------------------- ops
    def mpo(self, which: int):
        out = c_void_p()
        self._check(lib().qtt_mpo_get(self.h, which, byref(out)))
        return out

    def mpo_diff(self, axis: int, power: int = 1, dx: float = None):
        """A new derivative MPO handle (the context's stencil order); the
        caller frees it with free_mpo."""
        out = c_void_p()
        dx = self.params.L / self.N if dx is None else dx
        self._check(lib().qtt_mpo_diff(self.h, axis, power, dx, byref(out)))
        return out

    def free_mpo(self, m):
        lib().qtt_free_mpo(m)

    def apply_mpo(self, which, mps: MPS, eps=None, chi_max=None) -> MPS:
        """`which`: an operator index of qtt_mpo_get, or an MPO handle."""
        own = isinstance(which, int)
        m = self.mpo(which) if own else which
        out = c_void_p()
        try:
            self._check(lib().qtt_apply_mpo(self.h, m, mps.h,
                                            self.params.eps if eps is None else eps,
                                            self.params.chi_max if chi_max is None else chi_max,
                                            byref(out)))
        finally:
            if own:
                lib().qtt_free_mpo(m)
        return MPS(self, out.value)

    def add(self, coefs, terms, eps=None, chi_max=None) -> MPS:
        k = len(terms)
        cf = (c_double * k)(*coefs)
        hs = (c_void_p * k)(*[t.h.value for t in terms])
        out = c_void_p()
        self._check(lib().qtt_add(self.h, k, cf, hs, self.params.eps if eps is None else eps,
                                  self.params.chi_max if chi_max is None else chi_max,
                                  byref(out)))
        return MPS(self, out.value)

    def hadamard(self, a: MPS, b: MPS, eps=None, chi_max=None) -> MPS:
        out = c_void_p()
        self._check(lib().qtt_hadamard(self.h, a.h, b.h, self.params.eps if eps is None else eps,
                                       self.params.chi_max if chi_max is None else chi_max,
                                       byref(out)))
        return MPS(self, out.value)

    def compress(self, mps: MPS, eps=None, chi_max=None) -> MPS:
        self._check(lib().qtt_compress(self.h, mps.h, self.params.eps if eps is None else eps,
                                       self.params.chi_max if chi_max is None else chi_max))
        return mps

    def project(self, w1: MPS, w2: MPS, h: float, mu: float = None):
        """The penalty projection (qtt_project) with penalty mu (default: the
        context's)."""
        v1, v2 = c_void_p(), c_void_p()
        cg, sw = c_int(), c_int()
        st = lib().qtt_project(self.h, w1.h, w2.h, h, self.params.mu if mu is None else mu,
                               byref(v1), byref(v2), byref(cg), byref(sw))
        self._check(st, allow_not_converged=True)
        return MPS(self, v1.value), MPS(self, v2.value), cg.value, sw.value, st == 0

    def project_spectral(self, w1: MPS, w2: MPS):
        """The exact projection onto divergence-free fields (the penalty's
        mu -> infinity limit) through Fourier space, re-encoded to the
        context's (eps, chi_max): qtt_project_spectral."""
        v1, v2 = c_void_p(), c_void_p()
        self._check(lib().qtt_project_spectral(self.h, w1.h, w2.h, byref(v1), byref(v2)))
        return MPS(self, v1.value), MPS(self, v2.value)

    def rk4_step(self, u1: MPS, u2: MPS, dt: float, nu: float):
        """In place: u1, u2 receive the new state.  Returns True if every
        projection converged within its caps."""
        h1, h2 = c_void_p(u1.h.value), c_void_p(u2.h.value)
        st = lib().qtt_rk4_step(self.h, byref(h1), byref(h2), dt, nu)
        u1.h, u2.h = h1, h2
        self._check(st, allow_not_converged=True)
        return st == 0

    # -------------------------------------------------------- diagnostics
    def inner(self, a: MPS, b: MPS) -> float:
        """<a|b>, the sum over the grid of a(x) b(x)."""
        v = c_double()
        self._check(lib().qtt_inner(self.h, a.h, b.h, byref(v)))
        return v.value

    def fidelity(self, a: MPS, b: MPS) -> float:
        """|<a|b>|^2 / (<a|a> <b|b>) (Sec. III's fidelity of two states)."""
        ab, aa, bb = self.inner(a, b), self.inner(a, a), self.inner(b, b)
        return ab * ab / (aa * bb) if aa > 0 and bb > 0 else 0.0

    def tke_spectrum(self, u1: MPS, u2: MPS, kmax: int = None) -> np.ndarray:
        """E(k), k = 0..kmax (default: every shell of the grid), computed on
        the device (qtt_tke_spectrum)."""
        if kmax is None:
            kmax = int(np.ceil(self.N / np.sqrt(2.0))) + 1
        E = (c_double * (kmax + 1))()
        self._check(lib().qtt_tke_spectrum(self.h, u1.h, u2.h, kmax, E))
        return np.array(E[:])

    def kinetic_energy(self, u1: MPS, u2: MPS) -> float:
        """1/2 mean(u1^2 + u2^2) over the grid."""
        return 0.5 * (self.inner(u1, u1) + self.inner(u2, u2)) / float(self.N) ** 2

    def _step(self, fn, u1: MPS, u2: MPS, dt: float, nu: float):
        h1, h2 = c_void_p(u1.h.value), c_void_p(u2.h.value)
        st = fn(self.h, byref(h1), byref(h2), dt, nu)
        u1.h, u2.h = h1, h2
        self._check(st, allow_not_converged=True)
        return st == 0

    def euler_step(self, u1: MPS, u2: MPS, dt: float, nu: float):
        """Explicit Euler in place (App. B); True if the projection converged."""
        return self._step(lib().qtt_euler_step, u1, u2, dt, nu)

    def rk2_step(self, u1: MPS, u2: MPS, dt: float, nu: float):
        """Midpoint RK2 in place (App. B); True if both projections converged."""
        return self._step(lib().qtt_rk2_step, u1, u2, dt, nu)

    def gemm_tf32x3(self, A, B, transA: bool = False, transB: bool = False):
        """op(A) op(B) of FP64 device matrices on the tensor cores (3xTF32,
        FP32 accumulation); returns a new FP64 device tensor."""
        torch = _torch()
        A = A.contiguous()
        B = B.contiguous()
        M, K = (A.shape[1], A.shape[0]) if transA else (A.shape[0], A.shape[1])
        Kb, N = (B.shape[1], B.shape[0]) if transB else (B.shape[0], B.shape[1])
        if K != Kb:
            raise ValueError("inner dimensions differ")
        C = torch.empty((M, N), dtype=torch.float64, device=A.device)
        self._check(lib().qtt_gemm_tf32x3(self.h, M, N, K, c_void_p(A.data_ptr()), A.shape[1],
                                          int(transA), c_void_p(B.data_ptr()), B.shape[1],
                                          int(transB), c_void_p(C.data_ptr()), N))
        return C

    def gemm_ozaki(self, A, B, transA: bool = False, transB: bool = False, C=None,
                   alpha: float = 1.0, beta: float = 0.0):
        """alpha op(A) op(B) + beta C of FP64 device matrices (2-D, or 3-D
        batches along the first axis) on the BF16 tensor cores by the Ozaki
        splitting; returns C (a new tensor when C is None)."""
        torch = _torch()
        A = A.contiguous()
        B = B.contiguous()
        batched = A.dim() == 3
        A3 = A if batched else A.unsqueeze(0)
        B3 = B if batched else B.unsqueeze(0)
        nb = A3.shape[0]
        M, K = (A3.shape[2], A3.shape[1]) if transA else (A3.shape[1], A3.shape[2])
        Kb, N = (B3.shape[2], B3.shape[1]) if transB else (B3.shape[1], B3.shape[2])
        if K != Kb or B3.shape[0] != nb:
            raise ValueError("inner dimensions or batch counts differ")
        if C is None:
            C = torch.zeros((nb, M, N) if batched else (M, N), dtype=torch.float64,
                            device=A.device)
        C3 = C if batched else C.unsqueeze(0)
        if not C3.is_contiguous() or tuple(C3.shape) != (nb, M, N):
            raise ValueError("C must be a contiguous (batch,) M x N tensor")
        self._check(lib().qtt_gemm_ozaki(
            self.h, M, N, K, c_void_p(A3.data_ptr()), A3.shape[2], int(transA),
            A3.shape[1] * A3.shape[2], c_void_p(B3.data_ptr()), B3.shape[2], int(transB),
            B3.shape[1] * B3.shape[2], c_void_p(C3.data_ptr()), N, M * N, nb, float(alpha),
            float(beta)))
        return C

    def tc_stats(self):
        """(accepted, fell_back): the mixed form's tensor-core subspace
        searches, and those recomputed by the FP32 cluster SVD."""
        a, f = c_longlong(), c_longlong()
        self._check(lib().qtt_tc_stats(self.h, byref(a), byref(f)))
        return a.value, f.value

    def profile_begin(self):
        self._check(lib().qtt_profile_begin(self.h))

    def profile_end(self) -> dict:
        import json
        buf = ctypes.create_string_buffer(1 << 16)
        self._check(lib().qtt_profile_end(self.h, buf, len(buf)))
        return json.loads(buf.value.decode())

    def stats(self):
        a, b, c = c_longlong(), c_longlong(), c_longlong()
        self._check(lib().qtt_stats(self.h, byref(a), byref(b), byref(c)))
        return {"cg_iters": a.value, "sweeps": b.value, "launches": c.value}

    def graph_stats(self):
        """(stage graphs captured and kept, stage replays) of this context."""
        a, b = c_longlong(), c_longlong()
        self._check(lib().qtt_graph_stats(self.h, byref(a), byref(b)))
        return a.value, b.value

    # -------------------------------------------------- learned truncation
    def learned_set(self, params):
        """Install perceptron parameters (torch float32 tensor on the device)."""
        self._check(lib().qtt_learned_set(self.h, c_void_p(params.data_ptr())))

    def learned_next_step(self):
        self._check(lib().qtt_learned_next_step(self.h))

    def learned_log(self, max_slots: int = LEARNED_SLOTS):
        """(features [slots, n+1, 33], ranks [slots, n+1], slots used)."""
        nb = self.params.n + 1
        f = np.zeros((max_slots, nb, MLP_FEATURES), np.float32)
        r = np.zeros((max_slots, nb), np.int32)
        ns = c_int()
        self._check(lib().qtt_learned_log(self.h, c_void_p(f.ctypes.data), c_void_p(r.ctypes.data),
                                          max_slots, byref(ns)))
        return f, r, ns.value

    def learned_stats(self):
        a, b = c_longlong(), c_longlong()
        self._check(lib().qtt_learned_stats(self.h, byref(a), byref(b)))
        return a.value, b.value

    def rf_omega(self, key: int, D: int, w: int):
        torch = _torch()
        out = torch.empty((4 * D, w), dtype=torch.float64, device=f"cuda:{self.device}")
        self._check(lib().qtt_rf_omega(self.h, ctypes.c_ulonglong(key), D, w,
                                       c_void_p(out.data_ptr())))
        return out

    def mlp_forward(self, params, X):
        torch = _torch()
        out = torch.empty(X.shape[0], dtype=torch.float32, device=X.device)
        self._check(lib().qtt_mlp_forward(self.h, c_void_p(params.data_ptr()),
                                          c_void_p(X.data_ptr()), X.shape[0],
                                          c_void_p(out.data_ptr())))
        return out

    def mlp_loss_grad(self, params, X, y):
        torch = _torch()
        g = torch.empty(MLP_PARAMS, dtype=torch.float32, device=X.device)
        L = torch.empty(1, dtype=torch.float32, device=X.device)
        self._check(lib().qtt_mlp_loss_grad(self.h, c_void_p(params.data_ptr()),
                                            c_void_p(X.data_ptr()), c_void_p(y.data_ptr()),
                                            X.shape[0], c_void_p(g.data_ptr()),
                                            c_void_p(L.data_ptr())))
        return L, g

    def mlp_train(self, params, X, y, iters: int, lr: float):
        """Full-batch Adam in place on `params`; returns the loss before each step."""
        torch = _torch()
        losses = torch.empty(max(iters, 1), dtype=torch.float32, device=X.device)
        self._check(lib().qtt_mlp_train(self.h, c_void_p(params.data_ptr()),
                                        c_void_p(X.data_ptr()), c_void_p(y.data_ptr()),
                                        X.shape[0], iters, ctypes.c_float(lr),
                                        c_void_p(losses.data_ptr())))
        return losses[:iters]


class _BatchMember(Context):
    """A context owned by a Batch (created and destroyed by the library)."""

    def __init__(self, batch, handle, params, device):
        self.batch = batch        # the batch owns the C context: keep it alive
        self.device = device
        self.params = params
        self.h = c_void_p(handle)

    def close(self):
        self.h = c_void_p(None)   # the batch destroys it


class Batch:
    """B independent trajectories with their own parameters, stepped
    together by qtt_rk4_step_batched (one host thread per trajectory)."""

    def __init__(self, params_list, device: int = 0):
        B = len(params_list)
        arr = (Params * B)()
        for i, kw in enumerate(params_list):
            kw = dict(kw)
            arr[i] = Params(kw.pop("n"), kw.pop("L", 2 * np.pi), kw.pop("eps", 1e-8),
                            kw.pop("chi_max", 64), kw.pop("mu", 2.5e5), kw.pop("cg_tol", 1e-5),
                            kw.pop("cg_maxit", 100), kw.pop("sweep_tol", 1e-5),
                            kw.pop("max_sweeps", 20), kw.pop("precision", PREC_FP64),
                            kw.pop("learned_trunc", LEARNED_OFF), kw.pop("rf_oversample", 8),
                            kw.pop("rf_min_width", 128), kw.pop("graphs", 0),
                            kw.pop("fd_order", 0), kw.pop("rhs_form", 0),
                            kw.pop("projection", 0))
            if kw:
                raise TypeError(f"unknown parameters {sorted(kw)}")
        h = c_void_p()
        st = lib().qtt_batch_create(byref(h), device, B, arr)
        if st != 0:
            raise QttError(st, "qtt_batch_create failed")
        self.h = h
        self.contexts = [_BatchMember(self, lib().qtt_batch_context(h, i), arr[i], device)
                         for i in range(B)]

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            for c in getattr(self, "contexts", []):
                c.h = c_void_p(None)   # MPS of these contexts no longer free themselves
            lib().qtt_batch_destroy(self.h)
            self.h = c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def rk4_step(self, u1s, u2s, dts, nus):
        """In place on the MPS objects (u1s[i], u2s[i] of context i)."""
        B = len(self.contexts)
        a = (c_void_p * B)(*[m.h.value for m in u1s])
        b = (c_void_p * B)(*[m.h.value for m in u2s])
        st = lib().qtt_rk4_step_batched(self.h, a, b, (c_double * B)(*dts), (c_double * B)(*nus))
        for i in range(B):
            u1s[i].h, u2s[i].h = c_void_p(a[i]), c_void_p(b[i])
        if st not in (0, NOT_CONVERGED):
            raise QttError(st, "qtt_rk4_step_batched failed")
        return st == 0
