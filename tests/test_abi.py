"""CPU checks of the C ABI: the library builds, loads, exports every symbol
include/qtt.h declares, and the ctypes Params struct matches the header's
layout (no compute call: there is no GPU here)."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qtt.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(qtt_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2406_17823_b300 import build
    return build.build()


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    names = declared_functions()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name
    from paper_2406_17823_b300 import qtt
    assert sorted(qtt.EXPORTS) == names


def test_params_layout_matches_header():
    from paper_2406_17823_b300.qtt import Params
    prog = r"""
#include <stdio.h>
#include <stddef.h>
#include "qtt.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %d\n", sizeof(qtt_params),
         offsetof(qtt_params, n), offsetof(qtt_params, L), offsetof(qtt_params, eps),
         offsetof(qtt_params, chi_max), offsetof(qtt_params, mu), offsetof(qtt_params, cg_tol),
         offsetof(qtt_params, cg_maxit), offsetof(qtt_params, sweep_tol),
         offsetof(qtt_params, max_sweeps), offsetof(qtt_params, precision),
         offsetof(qtt_params, learned_trunc), offsetof(qtt_params, rf_oversample),
         offsetof(qtt_params, rf_min_width), offsetof(qtt_params, graphs),
         offsetof(qtt_params, fd_order), offsetof(qtt_params, rhs_form),
         offsetof(qtt_params, projection), QTT_MLP_PARAMS);
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "p.c")
        exe = os.path.join(d, "p")
        open(c, "w").write(prog)
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        got = list(map(int, subprocess.check_output([exe]).split()))
    from paper_2406_17823_b300.qtt import MLP_PARAMS
    from oracle.learned import N_PARAM
    want = [ctypes.sizeof(Params)] + [getattr(Params, f).offset for f, _ in Params._fields_]
    assert got == want + [MLP_PARAMS]
    assert MLP_PARAMS == N_PARAM


def test_null_arguments_are_rejected_without_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    lib.qtt_create.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    lib.qtt_create.restype = ctypes.c_int
    assert lib.qtt_create(None, 0, None, None) == 1  # QTT_ERR_ARG
    lib.qtt_destroy.argtypes = [ctypes.c_void_p]
    assert lib.qtt_destroy(None) == 1
    lib.qtt_last_error.restype = ctypes.c_char_p
    lib.qtt_last_error.argtypes = [ctypes.c_void_p]
    assert lib.qtt_last_error(None) == b"null context"


def test_newer_entry_points_reject_null_arguments_without_gpu(libpath):
    """Argument checks happen before any CUDA call: the learned-truncation,
    perceptron, batch, lower-order step, inner-product, graph-statistics and
    upload entry points all return QTT_ERR_ARG for null handles or pointers, on a
    machine without a GPU."""
    lib = ctypes.CDLL(libpath)
    vp = ctypes.c_void_p
    calls = [
        ("qtt_learned_set", [vp, vp], (None, None)),
        ("qtt_learned_next_step", [vp], (None,)),
        ("qtt_learned_stats", [vp, vp, vp], (None, None, None)),
        ("qtt_rf_omega", [vp, ctypes.c_ulonglong, ctypes.c_int, ctypes.c_int, vp], (None, 0, 1, 1, None)),
        ("qtt_mlp_forward", [vp, vp, vp, ctypes.c_int, vp], (None, None, None, 1, None)),
        ("qtt_mlp_loss_grad", [vp, vp, vp, vp, ctypes.c_int, vp, vp], (None,) * 4 + (1, None, None)),
        ("qtt_mlp_train", [vp, vp, vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_float, vp],
         (None,) * 4 + (1, 1, 1e-3, None)),
        ("qtt_batch_create", [vp, ctypes.c_int, ctypes.c_int, vp], (None, 0, 1, None)),
        ("qtt_batch_destroy", [vp], (None,)),
        ("qtt_rk4_step_batched", [vp, vp, vp, vp, vp], (None,) * 5),
        ("qtt_euler_step", [vp, vp, vp, ctypes.c_double, ctypes.c_double], (None, None, None, 1e-3, 0.0)),
        ("qtt_rk2_step", [vp, vp, vp, ctypes.c_double, ctypes.c_double], (None, None, None, 1e-3, 0.0)),
        ("qtt_inner", [vp, vp, vp, vp], (None,) * 4),
        ("qtt_graph_stats", [vp, vp, vp], (None,) * 3),
        ("qtt_mps_upload_packed", [vp, vp, vp, ctypes.c_int, vp], (None, None, None, 0, None)),
        ("qtt_tc_stats", [vp, vp, vp], (None,) * 3),
        ("qtt_tke_spectrum", [vp, vp, vp, ctypes.c_int, vp], (None, None, None, 4, None)),
        ("qtt_project_spectral", [vp, vp, vp, vp, vp], (None,) * 5),
        ("qtt_project", [vp, vp, vp, ctypes.c_double, ctypes.c_double, vp, vp, vp, vp],
         (None, None, None, 1e-3, 2.5e5, None, None, None, None)),
        ("qtt_mpo_diff", [vp, ctypes.c_int, ctypes.c_int, ctypes.c_double, vp],
         (None, 1, 1, 0.1, None)),
        ("qtt_gemm_tf32x3", [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, ctypes.c_int,
                             ctypes.c_int, vp, ctypes.c_int, ctypes.c_int, vp, ctypes.c_int],
         (None, 4, 4, 4, None, 4, 0, None, 4, 0, None, 4)),
        ("qtt_gemm_ozaki", [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, ctypes.c_int,
                            ctypes.c_int, ctypes.c_longlong, vp, ctypes.c_int, ctypes.c_int,
                            ctypes.c_longlong, vp, ctypes.c_int, ctypes.c_longlong, ctypes.c_int,
                            ctypes.c_double, ctypes.c_double],
         (None, 64, 64, 64, None, 64, 0, 0, None, 64, 0, 0, None, 64, 0, 1, 1.0, 0.0)),
    ]
    for name, argtypes, args in calls:
        f = getattr(lib, name)
        f.argtypes = argtypes
        f.restype = ctypes.c_int
        assert f(*args) == 1, name
    lib.qtt_batch_context.argtypes = [vp, ctypes.c_int]
    lib.qtt_batch_context.restype = vp
    assert lib.qtt_batch_context(None, 0) is None


def test_parameter_validation_without_gpu(libpath):
    """qtt_create checks its parameters before any CUDA call: out-of-range
    graph modes, learned-truncation modes and range-finder settings are
    QTT_ERR_ARG on a machine without a GPU."""
    from paper_2406_17823_b300.qtt import Params
    lib = ctypes.CDLL(libpath)
    lib.qtt_create.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    lib.qtt_create.restype = ctypes.c_int

    def params(**kw):
        p = Params(5, 6.283185307179586, 1e-8, 16, 2.5e5, 1e-5, 100, 1e-5, 20, 0, 0, 8, 128, 0, 0, 0, 0)
        for k, v in kw.items():
            setattr(p, k, v)
        return p

    bad = [dict(graphs=3), dict(graphs=-1), dict(learned_trunc=3), dict(precision=2),
           dict(learned_trunc=1, precision=1), dict(rf_oversample=257), dict(rf_min_width=0),
           dict(n=0), dict(n=16), dict(chi_max=0), dict(cg_maxit=0), dict(max_sweeps=0),
           dict(eps=-1.0), dict(L=0.0), dict(fd_order=3), dict(fd_order=10), dict(fd_order=-2), dict(rhs_form=2),
           dict(rhs_form=-1), dict(projection=2), dict(projection=-1),
           dict(projection=1, rhs_form=1), dict(projection=1, n=14)]
    h = ctypes.c_void_p()
    for kw in bad:
        p = params(**kw)
        assert lib.qtt_create(ctypes.byref(h), 0, None, ctypes.byref(p)) == 1, kw


def test_noalloc_size_checks_without_gpu(libpath):
    """qtt_to_dense_noalloc checks its sizes against the static array before
    any CUDA call: n outside 1..9 is QTT_ERR_ARG; at n = 9 a partial
    contraction 4^k D_k one column over 2^18 doubles is QTT_ERR_SHAPE, as are
    end bonds other than 1.  (The exact 2^18 edge is accepted and run in the
    GPU test.)"""
    lib = ctypes.CDLL(libpath)
    vp = ctypes.c_void_p
    f = lib.qtt_to_dense_noalloc
    f.argtypes = [vp, vp, ctypes.c_int, vp, vp]
    f.restype = ctypes.c_int
    fake = vp(16)  # never dereferenced: every case is rejected on the host

    def call(bonds, n):
        b = (ctypes.c_int * len(bonds))(*bonds)
        return f(fake, b, n, fake, None)

    edge = [1, 4, 16, 64, 64, 64, 64, 16, 4, 1]
    for k in (6, 7, 8):
        over = list(edge)
        over[k] += 1
        assert call(over, 9) == 2, k
    assert call([1] * 11, 10) == 1
    assert call([1] * 2, 0) == 1
    assert call([2, 4, 1], 2) == 2
    assert call([1, 0, 1], 2) == 2
    assert f(None, (ctypes.c_int * 3)(1, 4, 1), 2, fake, None) == 1
