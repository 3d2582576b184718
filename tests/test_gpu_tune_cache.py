"""The GEMM autotuner's choices persisted in a JSON file (QTT_TUNE_CACHE):
a first process tunes and writes them, a second one reads them, tunes
nothing new and reproduces the first one's result bit for bit.  And the
four FP64 GEMM tiles (QTT_GEMM_TILE forces one for every product) give the
same bits on a step of the implicit form, whose products span every tile's
shapes (small MPO cores over large batches, tall-skinny sweeps)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys, numpy as np
sys.path.insert(0, sys.argv[1])
import paper_2406_17823_b300 as P
import qtt_inputs as I
n = 7
ctx = P.Context(n, eps=1e-10, chi_max=32)
a = ctx.from_dense(I.random_field(n, seed=1) + 1e-3 * I.white_field(n, seed=2))
b = ctx.from_dense(I.random_field(n, seed=3))
out = ctx.hadamard(ctx.apply_mpo(1, a), b)
np.save(sys.argv[2], ctx.to_dense(out).cpu().numpy())
"""


def test_tune_cache_round_trip(tmp_path):
    cache = tmp_path / "tune.json"
    env = dict(os.environ, QTT_TUNE_CACHE=str(cache))
    r1 = subprocess.run([sys.executable, "-c", CHILD, ROOT, str(tmp_path / "a.npy")], env=env,
                        capture_output=True, text=True, timeout=300)
    assert r1.returncode == 0, r1.stderr[-2000:]
    first = json.loads(cache.read_text())
    assert first["version"] == 1 and len(first["entries"]) > 5
    assert all(len(e) == 8 and e[6] in (0, 1, 2, 3) and e[7] in (1, 2, 4, 8, 16)
               for e in first["entries"])
    r2 = subprocess.run([sys.executable, "-c", CHILD, ROOT, str(tmp_path / "b.npy")], env=env,
                        capture_output=True, text=True, timeout=300)
    assert r2.returncode == 0, r2.stderr[-2000:]
    assert json.loads(cache.read_text()) == first  # nothing new tuned
    assert np.array_equal(np.load(tmp_path / "a.npy"), np.load(tmp_path / "b.npy"))


CHILD_STEP = r"""
import sys, numpy as np
sys.path.insert(0, sys.argv[1])
import paper_2406_17823_b300 as P
import qtt_inputs as I
n = 7
(u, v), dx = I.shear_jet(n, seed=0)
ctx = P.Context(n, eps=1e-8, chi_max=24, rhs_form=P.RHS_IMPLICIT)
a, b = ctx.from_dense(u), ctx.from_dense(v)
ctx.rk4_step(a, b, 0.1 * dx / float(np.abs(u).max()), 1e-4)
np.save(sys.argv[2], np.stack([ctx.to_dense(a).cpu().numpy(), ctx.to_dense(b).cpu().numpy()]))
"""


def test_gemm_tiles_same_bits(tmp_path):
    outs = []
    for tile in range(4):
        env = dict(os.environ, QTT_GEMM_TILE=str(tile))
        f = tmp_path / f"t{tile}.npy"
        r = subprocess.run([sys.executable, "-c", CHILD_STEP, ROOT, str(f)], env=env,
                           capture_output=True, text=True, timeout=300)
        assert r.returncode == 0, r.stderr[-2000:]
        outs.append(np.load(f))
    assert np.all(np.isfinite(outs[0]))
    for t in range(1, 4):
        assert np.array_equal(outs[0], outs[t]), f"tile {t} differs from tile 0"
