"""bench.py's workload table on CPU: the configurations --workload selects,
their overrides, metric names and seeded initial states (no GPU)."""
import math
import os
import sys
import types

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def args(workload="jet", n=None, chi=None):
    return types.SimpleNamespace(workload=workload, n=n, chi=chi)


def test_default_is_the_headline_jet():
    w = bench.workload_of(args())
    assert (w["workload"], w["n"], w["chi_max"], w["eps"], w["Re"]) == (
        "shear_jet_2^10_chi64", 10, 64, 1e-8, 2e5)
    assert bench.metric_of(w) == bench.METRIC


def test_turbulence_and_taylor_green_configurations():
    t = bench.workload_of(args("turbulence"))
    assert (t["n"], t["chi_max"], t["eps"], t["Re"], t["k0"]) == (12, 128, 1e-7, 1e6, 10.0)
    assert bench.metric_of(t) == "RK4 steps/s at 2^12x2^12, chi=128"
    g = bench.workload_of(args("taylor_green"))
    assert (g["n"], g["chi_max"], g["eps"], g["Re"], g["dt"]) == (6, 16, 1e-12, 100.0, 1e-3)
    u, dx, dt = bench.workload_state(g, 0)
    assert dt == 1e-3 and math.isclose(dx, 2 * math.pi / 64)
    assert math.isclose(float(np.max(u[0])), 1.0, rel_tol=1e-3)


def test_overrides_rename_the_workload():
    w = bench.workload_of(args("turbulence", n=9, chi=32))
    assert (w["workload"], w["n"], w["chi_max"]) == ("turbulence_2^9_chi32", 9, 32)
    u, dx, dt = bench.workload_state(w, 5)
    assert u[0].shape == (512, 512)
    ke = 0.5 * float(np.mean(u[0] ** 2 + u[1] ** 2))
    assert math.isclose(ke, 1.0, rel_tol=1e-12)  # unit kinetic energy
    assert math.isclose(dt, 0.1 * dx / float(np.abs(u[0]).max()))
    u2, _, _ = bench.workload_state(w, 5)
    assert np.array_equal(u[0], u2[0])  # seeded
