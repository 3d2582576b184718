"""Benchmark: QTT RK4 steps per second on a 2^10 x 2^10 shear jet at chi = 64.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision all|both|mixed|fp64]
                    [--impl reference] [--batched B] [--eager | --stage-graphs] [--tight] [--rhs explicit|implicit]
                    [--projection penalty|spectral] [--workload jet|turbulence|taylor_green]
                    [--grid-bits n] [--chi c] [--no-cpu-baseline] [--no-e2e]
                    [--clocks-file PATH]

Workload (default): decaying double shear layer, periodic [0, 2 pi)^2 with
N = 2^10, u = tanh((y - pi/2)/delta) - tanh((y - 3 pi/2)/delta),
delta = 2 pi / 200, v = 0.05 sin x plus a seeded divergence-free
perturbation of RMS 1e-3 (seed 0); QTT with chi_max = 64, eps = 1e-8;
Re = 2e5; dt = 0.1 dx / max|u0|; the paper's solver settings (mu = 2.5e5,
CG tolerance 1e-5 with at most 100 iterations, sweep tolerance 1e-5).
A step is one full RK4 step (four penalised Euler minimisations) of both
velocity components; the state advances from step to step.

The metric compares the plain FP64 form with the mixed form.  By default
(--precision all) one run times four forms on the same initial state: W
warm-up steps of each, then K timed steps of each of
  * the mixed form with the paper's implicit right-hand side (the stages'
    nonlinear terms inside the projection's environments; FP64 products on
    the BF16 tensor cores by the Ozaki splitting, tensor-core subspace
    searches, FP64 factorisations): the line's value, ms_per_step, e2e and
    roofline;
  * the same scheme in FP64 (the line's "fp64_implicit" object);
  * the mixed form with the explicit right-hand side (B formed by zip-up
    Hadamard products; "mixed_explicit");
  * the explicit scheme in FP64 ("fp64").
All forms then take the same further steps (the profiled step, the e2e
steps), after which "mixed_vs_fp64_rel_l2" is the relative L2 distance of
the mixed and FP64 dense fields of the implicit scheme (both components),
"mixed_explicit_vs_fp64_rel_l2" that of the explicit scheme, and
"fp64_implicit_vs_fp64_rel_l2" that of the two FP64 schemes (different
truncations of the same equations, so of the order of the truncation
error, not of rounding).  --precision both times the explicit mixed and
FP64 forms, mixed | fp64 one explicit form only; with --rhs implicit the
named forms take the implicit right-hand side.  "oz_gemm" and "tc_gemm"
time the two tensor-core products alone.  --projection spectral replaces
every stage's penalty solve by the exact projection through Fourier space
(explicit right-hand side; with the default --precision the explicit mixed
and FP64 forms are timed).  --workload turbulence runs the decaying
turbulence configuration instead (2^12 x 2^12, chi 128, eps 1e-7, Re 1e6,
E(k) ~ k^4 exp(-2 (k/10)^2), unit kinetic energy), --workload taylor_green
the Taylor-Green vortex (2^6, chi 16, eps 1e-12, nu 0.01, dt 1e-3).

One JSON line is printed by rank 0.  With torchrun (N > 1) every rank runs
its own trajectory on its own GPU (replicas: the method has no exchange
step), value = all ranks' steps / the slowest rank's time.

--batched B steps B jets (seeds seed .. seed+B-1) together through the
batched C ABI (value = aggregate steps/s; one precision, mixed when "both").
By default every RK4 step is replayed as one CUDA graph (the projection's
CG and sweep loops as device-driven WHILE nodes), captured the second time
its shapes occur, so the warm-up steps capture and the timed steps replay;
--stage-graphs replays only the stages' right-hand sides, --eager launches
everything from the host; --tight runs CG and sweeps to 1e-12 (CG cap 500)
instead of the paper's settings; --grid-bits / --chi override n / chi_max
(smaller test cases).

CPU oracle: cpu_baseline times one whole RK4 step of the same workload
from its initial state with the oracle on one core (a subprocess with one
BLAS thread), in the scheme of the headline form (the paper's implicit step
by default; with the explicit forms in the run also one explicit step),
counting the algorithmic FLOPs of that step as it runs (matrix products
2MNK, Householder QR with explicit Q 4mn^2 - 4n^3/3, thin SVD
6mn^2 + 20n^3 for m >= n); every form's aggregate roofline uses the
explicit step's count as the unit of work per RK4 step (the oracle's
implicit step contracts the product MPOs literally, far more FLOPs than the
library's structured contraction).  --impl reference times the oracle as the reference arm in
the headline form's scheme: by default two consecutive whole implicit steps
(about a minute each), with --precision both | mixed | fp64 one untimed and
then min(K, 3) explicit steps (the line's "steps" is the number timed).

Timing: 3 warm-up steps by default, the L2 flushed (256 MB write) before
every timed step, CUDA events on the stepping stream (host clock between
device-wide synchronisations for a batch), SM clocks and throttle reasons
sampled during the timed regions; the roofline of the dominant kernel uses
the arithmetic it counts on the device, its launch times from one more step
under the library's launch profiler (outside the timed region) and a peak
measured in the same run.  gpu_launches counts the library's kernels run in
the timed region: kernels of a replayed graph once per replay, those of its
WHILE bodies once per pass (tallied on the device).  --clocks-file keeps
the clock samples.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RK4 steps/s at 2^10x2^10, chi=64"
WORKLOAD = dict(workload="shear_jet_2^10_chi64", n=10, chi_max=64, eps=1e-8, Re=2e5, mu=2.5e5,
                cg_tol=1e-5, cg_maxit=100, sweep_tol=1e-5, max_sweeps=20, seed=0,
                dt_rule="0.1*dx/max|u0|")
L2_FLUSH_BYTES = 256 << 20
# DRAM bytes (read + write) per launch of the dominant kernels, from one ncu
# capture of the widest launch at n = 8 (the same factor shapes as this
# workload; cold, serialised): profiles/ncu_k_svd_cluster_shear_jet_n8.md.
# To be re-taken whenever those kernels change.
NCU_TRAFFIC = {"k_svd_cluster": 520448 + 118272, "k_svd_cluster_f32": 8479232 + 444672}


# The other configurations of the workload table: the decaying turbulence
# (n = 12, chi = 128, eps = 1e-7, Re = 1e6, E(k) ~ k^4 exp(-2 (k/10)^2)) and the
# Taylor-Green vortex (n = 6, chi = 16, eps = 1e-12, nu = 0.01, dt = 1e-3).
WORKLOADS = {
    "jet": WORKLOAD,
    "turbulence": dict(WORKLOAD, workload="turbulence_2^12_chi128", n=12, chi_max=128, eps=1e-7,
                       Re=1e6, ic="turbulence", k0=10.0),
    "taylor_green": dict(WORKLOAD, workload="taylor_green_2^6_chi16", n=6, chi_max=16,
                         eps=1e-12, Re=100.0, ic="taylor_green", dt=1e-3, dt_rule="1e-3"),
}


def metric_of(w):
    if w["n"] == 10 and w["chi_max"] == 64:
        return METRIC
    return f"RK4 steps/s at 2^{w['n']}x2^{w['n']}, chi={w['chi_max']}"


def workload_of(args):
    """The workload of --workload with the --grid-bits / --chi overrides."""
    w = dict(WORKLOADS[args.workload])
    if args.n:
        w["n"] = args.n
    if args.chi:
        w["chi_max"] = args.chi
    if args.n or args.chi:
        w["workload"] = f"{w['workload'].split('_2^')[0]}_2^{w['n']}_chi{w['chi_max']}"
    return w


def workload_state(w, seed):
    """Initial velocity, grid spacing and time step of workload w (seeded)."""
    import qtt_inputs as I
    ic, n = w.get("ic", "jet"), w["n"]
    if ic == "turbulence":
        u, dx = I.decaying_turbulence(n, w["k0"], seed=seed)
    elif ic == "taylor_green":
        u, dx = I.taylor_green(n)
    else:
        u, dx = I.shear_jet(n, seed=seed)
    dt = w["dt"] if "dt" in w else 0.1 * dx / float(np.abs(u[0]).max())
    return u, dx, dt


def solver_kwargs(w):
    return dict(eps=w["eps"], chi_max=w["chi_max"], mu=w["mu"], cg_tol=w["cg_tol"],
                cg_maxit=w["cg_maxit"], sweep_tol=w["sweep_tol"], max_sweeps=w["max_sweeps"],
                projection=w.get("projection", 0))


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int, path: str = None):
        self.device = device
        self.proc = None
        self.path = path or os.path.join(tempfile.gettempdir(), f"qtt_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ peaks
def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            return json.load(open(path))
        except Exception:
            pass
    return {}


def gemm_peak(torch, dev, dtype):
    """ALU peak for the roofline denominator, measured in this run: cuBLAS
    GEMM 4096^3 in FP64 (DGEMM) or in FP32 with TF32 off (SGEMM on the FP32
    pipe); the measured-peaks file carries neither figure.  Best of 3."""
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    a = torch.randn(4096, 4096, device=dev, dtype=dtype)
    b = torch.randn(4096, 4096, device=dev, dtype=dtype)
    for _ in range(2):
        a @ b
    torch.cuda.synchronize()
    best = 1e9
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        a @ b
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1e3)
    del a, b
    torch.backends.cuda.matmul.allow_tf32 = prev
    return 2 * 4096 ** 3 / best / 1e12


# ------------------------------------------------------------------ CPU oracle
def oracle_steps(w, warm, timed):
    """Run the CPU oracle on the workload in a fresh interpreter whose BLAS is
    held to one thread: `warm` untimed RK4 steps from the initial state, then
    `timed` consecutive whole steps, each timed.  Returns the list of step
    times (s) and the algorithmic FLOPs of the timed steps (per step)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1",
               MKL_NUM_THREADS="1", CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-steps",
                        json.dumps(dict(w, warm=warm, timed=timed))], env=env,
                       capture_output=True, text=True, timeout=1800)
    if r.returncode != 0:
        raise RuntimeError("oracle timing failed:\n" + r.stderr[-2000:])
    out = json.loads(r.stdout.strip().splitlines()[-1])
    return out["times"], out["flops"]


class FlopCounter:
    """Counts the algorithmic FLOPs of numpy's contraction and factorisation
    calls while installed (the oracle's matrix products go through
    tensordot / einsum / matmul; its factorisations through linalg.qr and
    linalg.svd).  Models: a product 2 x (output size) x (contracted size);
    Householder QR with explicit Q 4mn^2 - 4n^3/3 (m >= n); thin SVD
    6mn^2 + 20n^3 (R-SVD, U_1, Sigma and V; m >= n)."""

    def __init__(self):
        self.total = 0.0
        self._saved = []

    def install(self):
        import numpy
        import numpy.linalg
        c = self

        def wrap(mod, name, count):
            orig = getattr(mod, name)

            def f(*a, **k):
                out = orig(*a, **k)
                c.total += count(out, *a, **k)
                return out
            self._saved.append((mod, name, orig))
            setattr(mod, name, f)

        def td(out, A, B, axes=2, **_):
            A, B = numpy.asarray(A), numpy.asarray(B)
            if isinstance(axes, int):
                kdims = A.shape[A.ndim - axes:]
            else:
                ax = axes[0] if isinstance(axes[0], (list, tuple)) else [axes[0]]
                kdims = [A.shape[i] for i in ax]
            return 2.0 * numpy.asarray(out).size * float(numpy.prod(kdims))

        def ein(out, spec, *ops, **_):
            # every index of a two-operand contraction appears once in the loop nest
            ins = spec.split("->")[0].split(",")
            ext = {}
            for sub, op in zip(ins, ops):
                for ch, n in zip(sub, numpy.shape(op)):
                    ext[ch] = n
            return 2.0 * float(numpy.prod(list(ext.values()))) if len(ops) > 1 else 0.0

        def mm(out, A, B, **_):
            A = numpy.asarray(A)
            return 2.0 * numpy.asarray(out).size * A.shape[-1]

        def qr(out, A, *a, **k):
            m, n = numpy.shape(A)[-2:]
            m, n = max(m, n), min(m, n)
            return 4.0 * m * n * n - 4.0 / 3.0 * n ** 3

        def svd(out, A, *a, **k):
            m, n = numpy.shape(A)[-2:]
            m, n = max(m, n), min(m, n)
            return 6.0 * m * n * n + 20.0 * n ** 3

        wrap(numpy, "tensordot", td)
        wrap(numpy, "einsum", ein)
        wrap(numpy, "matmul", mm)
        wrap(numpy.linalg, "qr", qr)
        wrap(numpy.linalg, "svd", svd)
        return self

    def uninstall(self):
        for mod, name, orig in reversed(self._saved):
            setattr(mod, name, orig)
        self._saved = []


def _oracle_steps_child(wjson):
    w = json.loads(wjson)
    counter = FlopCounter().install()  # before the oracle binds numpy's functions
    from oracle import qtt as Q
    u, dx, dt = workload_state(w, w["seed"])
    p = Q.Params(eps=w["eps"], chi_max=w["chi_max"], mu=w["mu"], cg_tol=w["cg_tol"],
                 cg_maxit=w["cg_maxit"], sweep_tol=w["sweep_tol"], max_sweeps=w["max_sweeps"],
                 projection="spectral" if w.get("projection", 0) == 1 else "penalty")
    uq = [Q.from_dense(f, p.eps, p.chi_max) for f in u]
    ops = Q.build_operators(w["n"], dx)
    nu = 1.0 / w["Re"]
    # the scheme of the form it stands beside: the explicit step (B formed)
    # or the paper's implicit one
    step = Q.rk4_step_implicit if w.get("rhs_form", 0) == 1 else Q.rk4_step
    for _ in range(w["warm"]):
        uq = step(uq, dt, nu, p, ops)
    times, flops = [], []
    for _ in range(w["timed"]):
        f0 = counter.total
        t = time.perf_counter()
        uq = step(uq, dt, nu, p, ops)
        times.append(time.perf_counter() - t)
        flops.append(counter.total - f0)
    print(json.dumps({"times": times, "flops": flops}))


# ------------------------------------------------------------------ ranks
def reduce_max_time(t_local, dist=None, device="cpu"):
    """The timed region of a multi-rank run: the maximum over ranks of each
    rank's own time (seconds); the local time when there is one rank."""
    if dist is None:
        return t_local
    import torch
    tt = torch.tensor([t_local], device=device, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w = workload_of(args)
    # the scheme of the main arm's headline form: the paper's implicit step
    # by default (an implicit oracle step takes about a minute on one core,
    # so two steps and no untimed one), the explicit step for the explicit
    # precisions
    implicit = (args.precision == "all" or args.rhs == "implicit") and \
        args.projection != "spectral"
    if args.projection == "spectral":
        w["projection"] = 1
        w["workload"] += "_spectral_projection"
    if implicit:
        w["rhs_form"] = 1
        w["workload"] += "_implicit_rhs"
    warm = 0 if implicit else 1
    timed = max(1, min(args.steps, 2 if implicit else 3))
    times, flops = oracle_steps(w, warm, timed)
    total = sum(times)
    value = timed / total
    line = {"impl": "reference", "metric": metric_of(w), "value": value, "unit": "steps/s",
            "n_gpus": args.gpus, "steps": timed, "steps_requested": args.steps,
            "warmup": warm, "ms_per_step": 1e3 * total / timed, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {**w, "parallelism": "none (CPU oracle)"},
            "algorithmic_flops_per_step": statistics.mean(flops),
            "cpu_baseline": {"value": value, "unit": "steps/s", "cores": 1, "kind": "oracle",
                             "sample": (f"{warm} untimed and {timed} consecutive whole RK4 "
                                        "steps of the workload ("
                                        + ("the paper's implicit scheme" if implicit else
                                           "explicit scheme") + "), timed; numpy FP64 oracle on "
                                        "one BLAS thread")},
            "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ main arm
def make_form(P, w, prec, graphs, B, local, rank, rhs_form=None):
    """Contexts and initial states of one form (same seeds for every form)."""
    rhs = w.get("rhs_form", 0) if rhs_form is None else rhs_form
    B = max(1, B)
    if B > 1:
        batch = P.Batch([dict(n=w["n"], precision=prec, graphs=graphs,
                              rhs_form=rhs, **solver_kwargs(w))
                         for _ in range(B)], device=local)
        ctxs = batch.contexts
    else:
        batch = None
        ctxs = [P.Context(w["n"], precision=prec, device=local, graphs=graphs,
                          rhs_form=rhs, **solver_kwargs(w))]
    states, dts = [], []
    for i, c in enumerate(ctxs):
        u, dx, dt_i = workload_state(w, w["seed"] + rank * B + i)
        states.append([c.from_dense(f) for f in u])
        dts.append(dt_i)
    nu = 1.0 / w["Re"]

    def step():
        if B > 1:
            return batch.rk4_step([s[0] for s in states], [s[1] for s in states], dts, [nu] * B)
        return ctxs[0].rk4_step(states[0][0], states[0][1], dts[0], nu)

    return dict(batch=batch, ctxs=ctxs, states=states, step=step, B=B)


def time_steps(torch, form, K, flush):
    """K timed steps: L2 flushed before each, CUDA events on the stepping
    stream (host clock between device-wide synchronisations for a batch)."""
    step, B = form["step"], form["B"]
    times, converged = [], True
    launches0 = sum(c.stats()["launches"] for c in form["ctxs"])
    replays0 = sum(c.graph_stats()[1] for c in form["ctxs"])
    tc0 = [c.tc_stats() for c in form["ctxs"]]
    for _ in range(K):
        flush.zero_()  # evict the L2 between timed steps
        if B > 1:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            converged &= step()
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
        else:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            converged &= step()
            e1.record()
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
    torch.cuda.synchronize()
    launches = sum(c.stats()["launches"] for c in form["ctxs"]) - launches0
    replays = sum(c.graph_stats()[1] for c in form["ctxs"]) - replays0
    tc1 = [c.tc_stats() for c in form["ctxs"]]
    tc = {"accepted": sum(b[0] - a[0] for a, b in zip(tc0, tc1)),
          "fell_back": sum(b[1] - a[1] for a, b in zip(tc0, tc1))}
    return times, bool(converged), launches, replays, tc


def profile_step(torch, form):
    """Per-kernel device times: one more step under the launch profiler (CUDA
    events around every launch, which also makes the stages launch eagerly),
    outside the timed region."""
    ctx = form["ctxs"][0]
    ctx.profile_begin()
    form["step"]()
    torch.cuda.synchronize()
    return ctx.profile_end()


def e2e_steps(torch, form, n_steps, flush, world):
    """The same metric through the C ABI with host buffers: upload the packed
    states from host memory (into the state objects, whose capacities the
    step graphs are keyed on), one step, download the packed results."""
    ctxs, states = form["ctxs"], form["states"]
    cores = [[c.to_cores(x) for x in st] for c, st in zip(ctxs, states)]
    times, h2d, d2h = [], 0, 0
    for _ in range(n_steps):
        host = cores
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for c, st, hc in zip(ctxs, states, host):
            for x, cc in zip(st, hc):
                c.upload_cores(x, cc)
        form["step"]()
        out = [[c.to_cores(x) for x in st] for c, st in zip(ctxs, states)]
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
        h2d = sum(a.nbytes for hc in host for cc in hc for a in cc)
        d2h = sum(a.nbytes for oc in out for cc in oc for a in cc)
        cores = out
    value = world * form["B"] * len(times) / sum(times) if times else None
    return {"value": value, "unit": "steps/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h}


OZ_PAIRS = 36  # slice products of the Ozaki splitting per FP64 product (8 slices, p + q <= 7)
# ncu dram__bytes_read.sum + dram__bytes_write.sum of one 12288 x 256 x 64 launch
# (profiles/ncu_k_gemm_oz_12288x256x64.md): the operands read once, C stays in L2
OZ_NCU_TRAFFIC = 6783488 + 272384


def roofline_of(torch, dev, prof):
    """Roofline of the kernel with the largest share of device time."""
    dom, rec = max(prof.items(), key=lambda kv: kv[1]["ms"])
    tot_ms = sum(v["ms"] for v in prof.values())
    if dom.startswith("k_gemm_oz"):
        # FP64 products on the BF16 tensor cores: the scheme's BF16 slice
        # products against the sustained BF16 peak (a kernel inside a long
        # step); the FP64-equivalent rate against DGEMM beside it
        peaks = measured_peaks()
        bf16 = peaks.get("bf16_tflops_sustained") or peaks.get("bf16_tflops")
        avg_ms = rec["ms"] / rec["launches"]
        fpl = rec["flops"] / rec["launches"]
        f64eq = fpl / (avg_ms * 1e-3) / 1e12
        achieved = OZ_PAIRS * f64eq
        dpk = gemm_peak(torch, dev, torch.float64)
        return {"kernel": dom, "bound": "tensor", "achieved": achieved,
                "peak": bf16, "unit": "TFLOP/s", "frac": achieved / bf16 if bf16 else None,
                "traffic": None,
                "traffic_source": "null: this kernel's launches span many product shapes; the "
                                  "ncu DRAM bytes of the projection's 12288 x 256 x 64 launch "
                                  "are in oz_gemm (profiles/ncu_k_gemm_oz_12288x256x64.md)",
                "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained (of measured)",
                "achieved_source": f"{OZ_PAIRS} BF16 slice products per FP64 product "
                                   "(algorithmic 2MNK each) / launch time",
                "fp64_equivalent_tflops": f64eq, "fp64_dgemm_peak": dpk,
                "fp64_equivalent_over_dgemm": f64eq / dpk if dpk else None,
                "share_of_device_time": rec["ms"] / tot_ms if tot_ms else None,
                "launches_timed": rec["launches"], "avg_launch_ms": avg_ms,
                "flops_per_launch": fpl,
                "timing_source": "one step after the timed region, launched eagerly under the "
                                 "library's launch profiler",
                "kernel_shares": {k: round(v["ms"] / tot_ms, 4) for k, v in prof.items()}}
    # the dominant kernel's arithmetic type decides the pipe it is bound by:
    # the FP32 subspace search of the mixed form runs on the FP32 pipe
    f32_kernel = dom.endswith("_f32")
    peak = gemm_peak(torch, dev, torch.float32 if f32_kernel else torch.float64)
    avg_ms = rec["ms"] / rec["launches"]
    flops_per_launch = rec["flops"] / rec["launches"]
    achieved = flops_per_launch / (avg_ms * 1e-3) / 1e12
    cluster = dom.startswith("k_svd_cluster")
    return {"kernel": dom, "bound": "alu",
            "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak if peak else None,
            "traffic": NCU_TRAFFIC.get(dom),
            "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of the widest "
                              "launch (factor 256 wide) at n = 8, same shapes; see profiles/",
            "peak_source": ("FP32 cuBLAS SGEMM (TF32 off) 4096^3" if f32_kernel else
                            "FP64 cuBLAS DGEMM 4096^3") + " measured in this run (of measured)",
            # one launch of the cluster SVD holds a 16-CTA cluster (16 of the 148 SMs)
            "cluster_sms": 16 if cluster else None,
            "frac_of_cluster_peak": achieved / (peak * 16 / 148) if peak and cluster else None,
            "flops_source": ("counted on the device (QR, Jacobi dots and rotations, Q "
                             "application)" if cluster else "host model"),
            "share_of_device_time": rec["ms"] / tot_ms if tot_ms else None,
            "launches_timed": rec["launches"], "avg_launch_ms": avg_ms,
            "flops_per_launch": flops_per_launch,
            "timing_source": "one step after the timed region, launched eagerly under the "
                             "library's launch profiler",
            "kernel_shares": {k: round(v["ms"] / tot_ms, 4) for k, v in prof.items()}}


def tc_gemm_record(torch, ctx, peaks):
    """Throughput of the tensor-core product (qtt_gemm_tf32x3: 3xTF32 on
    tcgen05, FP32 accumulation) at 4096^3, CUDA events over 5 calls after
    3 warm-up calls: the whole call (operand split, product, reduction)
    and the product kernel alone (from the launch profiler).  Peak: the
    measured BF16 tensor peak x 1/2 (TF32 runs at half the BF16 rate),
    counting the three TF32 products of each 3xTF32 step."""
    n = 4096
    A = torch.randn(n, n, dtype=torch.float64, device="cuda")
    B = torch.randn(n, n, dtype=torch.float64, device="cuda")
    for _ in range(3):
        ctx.gemm_tf32x3(A, B)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(5):
        ctx.gemm_tf32x3(A, B)
    e1.record()
    e1.synchronize()
    call_ms = e0.elapsed_time(e1) / 5
    ctx.profile_begin()
    ctx.gemm_tf32x3(A, B)
    torch.cuda.synchronize()
    kms = ctx.profile_end()["k_tc_gemm"]["ms"]
    flops = 2.0 * n ** 3
    tf32_peak = peaks.get("bf16_tflops") / 2 if peaks.get("bf16_tflops") else None
    tensor_tflops = 3 * flops / (kms * 1e-3) / 1e12
    return {"shape": [n, n, n], "call_ms": call_ms, "kernel_ms": kms,
            "algorithmic_tflops": flops / (kms * 1e-3) / 1e12,
            "tensor_tflops": tensor_tflops, "tf32_peak_tflops": tf32_peak,
            "frac": tensor_tflops / tf32_peak if tf32_peak else None,
            "peak_source": "MEASURED_PEAKS.json bf16_tflops x 1/2 (TF32 / BF16 nominal ratio; "
                           "of measured)"}


def oz_gemm_record(torch, ctx, peaks):
    """Throughput of the emulated FP64 product (qtt_gemm_ozaki: eight BF16
    slices per K chunk of 64 on tcgen05, exact FP32 accumulation, one FP64
    rounding) at the projection's dominant shape and at a large K = 64
    shape: CUDA events over 10 calls after 3 warm-up calls."""
    out = []
    for (M, N, K) in ((12288, 256, 64), (16384, 4096, 64)):
        A = torch.randn(M, K, dtype=torch.float64, device="cuda")
        B = torch.randn(K, N, dtype=torch.float64, device="cuda")
        C = torch.empty(M, N, dtype=torch.float64, device="cuda")
        for _ in range(3):
            ctx.gemm_ozaki(A, B, C=C)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(10):
            ctx.gemm_ozaki(A, B, C=C)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1) / 10
        f64eq = 2.0 * M * N * K / (ms * 1e-3) / 1e12
        bf16 = peaks.get("bf16_tflops")
        rec = {"shape": [M, N, K], "ms": ms, "fp64_equivalent_tflops": f64eq,
               "tensor_tflops": OZ_PAIRS * f64eq, "bf16_peak_tflops": bf16,
               "frac": OZ_PAIRS * f64eq / bf16 if bf16 else None,
               "algorithmic_bytes": 8 * (M * K + K * N + M * N)}
        if (M, N, K) == (12288, 256, 64):
            rec["ncu_dram_bytes"] = OZ_NCU_TRAFFIC
        out.append(rec)
    return {"shapes": out, "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst; of measured)"}


def rel_l2(fa, fb):
    """sqrt(sum_i |a_i - b_i|^2) / sqrt(sum_i |b_i|^2) over the components."""
    num = sum(float(((a - b) ** 2).sum()) for a, b in zip(fa, fb))
    den = sum(float((b ** 2).sum()) for b in fb)
    return math.sqrt(num / den) if den > 0 else None


def run_ensemble(args):
    """Ragged ensemble of K independent trajectories stepped together by
    qtt_rk4_step_batched (one context, stream set and host thread each, every
    RK4 step of a trajectory replayed as a CUDA graph): trajectory t has
    n = 8 + (t mod 5), chi_max = (16, 32, 64, 128)[(t div 5) mod 4], the
    random-phase turbulence initial condition E(k) ~ k^4 exp(-2 (k/10)^2)
    with seed t, eps = 1e-7, Re = 1e6, dt = 0.1 dx / max|u0|, the paper's
    solver settings, mixed form.  value = K x steps / time (aggregate RK4
    steps per second); --ensemble-sequential also times one step of every
    trajectory on its own (the same contexts, one after another)."""
    import torch
    import paper_2406_17823_b300 as P
    import qtt_inputs as I
    K = args.ensemble
    torch.cuda.set_device(0)
    dev = torch.device("cuda:0")
    prec = P.PREC_FP64 if args.precision == "fp64" else P.PREC_MIXED
    plist, states, dts = [], [], []
    for t in range(K):
        n = 8 + t % 5
        chi = (16, 32, 64, 128)[(t // 5) % 4]
        plist.append(dict(n=n, eps=1e-7, chi_max=chi, precision=prec, graphs=2))
    batch = P.Batch(plist, device=0)
    for t, c in enumerate(batch.contexts):
        u, dx = I.decaying_turbulence(plist[t]["n"], k0=10, seed=t)
        states.append([c.from_dense(f) for f in u])
        dts.append(0.1 * dx / float(max(np.abs(u[0]).max(), np.abs(u[1]).max())))
    nus = [1e-6] * K
    step = lambda: batch.rk4_step([s_[0] for s_ in states], [s_[1] for s_ in states], dts, nus)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    times = []
    with ClockSampler(0, args.clocks_file) as clk:
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            step()
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
    total = sum(times)
    seq = None
    if args.ensemble_sequential:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for c, st, dt in zip(batch.contexts, states, dts):
            c.rk4_step(st[0], st[1], dt, 1e-6)
        torch.cuda.synchronize()
        seq = K / (time.perf_counter() - t0)
    bonds = [max(s_[0].bonds) for s_ in states]
    line = {"metric": "aggregate RK4 steps/s, ragged turbulence ensemble", "value": K * args.steps / total,
            "unit": "steps/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if prec == P.PREC_FP64 else "tf32x3/f32/f64",
            "data": "synthetic (seeded turbulence initial conditions)",
            "config": {"workload": f"turbulence_ensemble_x{K}", "trajectories": K,
                       "n": "8 + (t mod 5)", "chi_max": "(16, 32, 64, 128)[(t div 5) mod 4]",
                       "eps": 1e-7, "Re": 1e6, "k0": 10, "seeds": f"0..{K - 1}",
                       "precision": args.precision, "step_graphs": True,
                       "l2": "flushed between timed steps (256 MB write)"},
            "sequential_steps_per_s": seq, "max_bond_after": max(bonds),
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="own")
    ap.add_argument("--precision", default="all", choices=["all", "both", "fp64", "mixed"],
                    help="all (default): the mixed form (the line's value), the FP64 form and "
                         "the paper's implicit form in FP64; both: the first two")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer pass")
    ap.add_argument("--workload", default="jet", choices=sorted(WORKLOADS),
                    help="jet (default): the 2^10 shear jet at chi 64; turbulence: decaying "
                         "turbulence at 2^12, chi 128, eps 1e-7, Re 1e6; taylor_green: 2^6, "
                         "chi 16, eps 1e-12, nu 0.01, dt 1e-3")
    ap.add_argument("--grid-bits", "--n", dest="n", type=int, default=None,
                    help="override grid bits (testing only; under torchrun use --grid-bits)")
    ap.add_argument("--tight", action="store_true",
                    help="CG and sweep tolerances 1e-12, CG cap 500, instead of the paper's "
                         "1e-5 / 1e-5 / 100")
    ap.add_argument("--batched", type=int, default=1,
                    help="B > 1: B trajectories (seeds seed..seed+B-1) stepped together by "
                         "qtt_rk4_step_batched; value = aggregate steps/s")
    ap.add_argument("--chi", type=int, default=None, help="override chi_max (testing only)")
    ap.add_argument("--eager", action="store_true", help="launch every kernel from the host")
    ap.add_argument("--clocks-file", default=None,
                    help="where the nvidia-smi clock samples of the timed region go (CSV; "
                         "default: a file in the temporary directory)")
    ap.add_argument("--rhs", default="explicit", choices=["explicit", "implicit"],
                    help="the stages' right-hand side: formed as an MPS (explicit) or the "
                         "paper's form inside the projection (implicit)")
    ap.add_argument("--projection", default="penalty", choices=["penalty", "spectral"],
                    help="each stage's projection: the paper's penalty solve or the exact "
                         "projection through Fourier space (explicit right-hand side only)")
    ap.add_argument("--stage-graphs", action="store_true",
                    help="replay only each stage's right-hand side as a CUDA graph (the "
                         "projection launched from the host)")
    ap.add_argument("--ensemble", type=int, default=0,
                    help="K > 0: the ragged turbulence ensemble of K trajectories (n, chi per "
                         "trajectory) through the batched C ABI instead of the jet")
    ap.add_argument("--ensemble-sequential", action="store_true",
                    help="with --ensemble: also time one step of each trajectory alone")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.ensemble > 0:
        return run_ensemble(args)

    import torch
    import paper_2406_17823_b300 as P

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    w = workload_of(args)
    if args.tight:
        w.update(cg_tol=1e-12, sweep_tol=1e-12, cg_maxit=500)
        w["workload"] += "_tight"
    graphs = 0 if args.eager else (1 if args.stage_graphs else 2)
    if args.rhs == "implicit":
        w["rhs_form"] = 1
        w["workload"] += "_implicit_rhs"
    if args.projection == "spectral":
        if args.rhs == "implicit":
            ap.error("--projection spectral needs the explicit right-hand side")
        w["projection"] = 1
        w["workload"] += "_spectral_projection"
    B = max(1, args.batched)
    if B > 1:
        w["workload"] = f"{w['workload']}_x{B}_trajectories"
    names = {"all": ["mixed_implicit", "fp64_implicit", "mixed", "fp64"],
             "both": ["mixed", "fp64"], "mixed": ["mixed"], "fp64": ["fp64"]}[args.precision]
    if B > 1 or args.rhs == "implicit":
        names = ["mixed"] if args.precision in ("all", "both") else names
    if args.projection == "spectral" and args.precision == "all":
        names = ["mixed", "fp64"]  # the implicit forms have no spectral projection
    precs = {"mixed": P.PREC_MIXED, "fp64": P.PREC_FP64, "fp64_implicit": P.PREC_FP64,
             "mixed_implicit": P.PREC_MIXED}
    rhs_of = {"fp64_implicit": P.RHS_IMPLICIT, "mixed_implicit": P.RHS_IMPLICIT}
    forms = {nm: make_form(P, w, precs[nm], graphs, B, local, rank, rhs_of.get(nm))
             for nm in names}
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    for nm in names:
        for _ in range(args.warmup):
            forms[nm]["step"]()
    barrier()
    res = {}
    with ClockSampler(local, args.clocks_file) as clk:
        for nm in names:
            barrier()
            wall0 = time.perf_counter()
            times, conv, launches, replays, tc = time_steps(torch, forms[nm], args.steps, flush)
            barrier()
            t_max = reduce_max_time(sum(times), dist, dev)
            res[nm] = dict(t_max=t_max, converged=conv, launches=launches, replays=replays,
                           wall=time.perf_counter() - wall0, tc=tc)
    for nm in names:
        res[nm]["prof"] = profile_step(torch, forms[nm])
    n_e2e = 0 if args.no_e2e else max(1, min(args.steps, 2))
    head = names[0]
    e2e = e2e_steps(torch, forms[head], n_e2e, flush, world)
    for nm in names[1:]:  # the same number of steps, so the states can be compared
        for _ in range(n_e2e):
            forms[nm]["step"]()
    torch.cuda.synchronize()
    cmp = cmp_imp = cmp_mi = None
    if len(names) > 1:
        fields = {nm: [forms[nm]["ctxs"][0].to_dense(x).cpu().numpy()
                       for x in forms[nm]["states"][0]] for nm in names}
        if "mixed" in names and "fp64" in names:
            cmp = rel_l2(fields["mixed"], fields["fp64"])
        if "fp64_implicit" in names and "fp64" in names:
            cmp_imp = rel_l2(fields["fp64_implicit"], fields["fp64"])
        if "mixed_implicit" in names and "fp64_implicit" in names:
            cmp_mi = rel_l2(fields["mixed_implicit"], fields["fp64_implicit"])
    steps_taken = args.warmup + args.steps + 1 + n_e2e

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    def summary(nm):
        r = res[nm]
        return {"value": world * B * args.steps / r["t_max"],
                "ms_per_step": 1e3 * r["t_max"] / args.steps,
                "gpu_launches": r["launches"], "step_graph_replays_timed": r["replays"],
                "all_projections_converged": r["converged"], "wall_s": r["wall"],
                "tc_subspace_searches_timed": r["tc"],
                "roofline": roofline_of(torch, dev, r["prof"])}

    sums = {nm: summary(nm) for nm in names}
    cpu, oracle_flops = None, {}
    if not args.no_cpu_baseline:
        # one oracle step of each scheme timed: the headline form's scheme
        # gives cpu_baseline; both give the algorithmic FLOPs per step of
        # their forms' aggregate rooflines
        schemes = sorted({0} | {1 if (nm.endswith("implicit") or w.get("rhs_form", 0) == 1)
                                else 0 for nm in names})
        ostep = {}
        for sch in schemes:
            times, flops = oracle_steps(dict(w, rhs_form=sch), 0, 1)
            ostep[sch] = (times[0], flops[0])
        oracle_flops = {sch: ostep[sch][1] for sch in schemes}
        hsch = 1 if (head.endswith("implicit") or w.get("rhs_form", 0) == 1) else 0
        cpu = {"value": 1.0 / ostep[hsch][0], "unit": "steps/s", "cores": 1, "kind": "oracle",
               "sample": "one whole RK4 step of the same workload from its initial state ("
                         + ("the paper's implicit scheme, as the headline form" if hsch else
                            "explicit scheme") + "), numpy FP64 oracle on one BLAS thread",
               "algorithmic_flops_per_step": ostep[hsch][1]}
        if hsch:
            cpu["explicit_scheme"] = {"value": 1.0 / ostep[0][0],
                                      "algorithmic_flops_per_step": ostep[0][1]}
            cpu["flops_note"] = ("the oracle's implicit step contracts the product MPOs H_b D_j "
                                 "literally; the library's structured contraction does about a "
                                 "quarter of those FLOPs")
    fp64_peak = None
    for nm in names:
        rf = sums[nm]["roofline"]
        if rf["peak_source"].startswith("FP64"):
            fp64_peak = rf["peak"]
    if oracle_flops:
        if fp64_peak is None:
            fp64_peak = gemm_peak(torch, dev, torch.float64)
        # one unit of work per RK4 step for every form: the explicit scheme's
        # count (the oracle's implicit step contracts the 3 chi-bond product
        # MPOs literally, about 9x the explicit step's FLOPs and about 4x what
        # the library's structured contraction does, so its count is no
        # measure of the work the GPU forms do)
        unit = oracle_flops.get(0)
        for nm in names:
            if unit is None:
                break
            ach = unit * sums[nm]["value"] / world / B / 1e12
            sums[nm]["roofline"]["aggregate"] = {
                "flops_per_step": unit, "achieved": ach, "unit": "TFLOP/s",
                "peak": fp64_peak, "frac": ach / fp64_peak,
                "source": "algorithmic FLOPs of one RK4 step of the explicit scheme counted in "
                          "the CPU oracle (FP64 algorithm), a common unit of work per step for "
                          "every form, x steps/s; peak = FP64 cuBLAS DGEMM measured in this run "
                          "(of measured)"}
    clocks = clk.summary()
    peaks = measured_peaks()
    tcg = ozg = None
    mixed_nm = next((nm for nm in names if nm.startswith("mixed")), None)
    if mixed_nm:
        tcg = tc_gemm_record(torch, forms[mixed_nm]["ctxs"][0], peaks)
        ozg = oz_gemm_record(torch, forms[mixed_nm]["ctxs"][0], peaks)
    hs = sums[head]
    line = {"metric": metric_of(w), "value": hs["value"], "unit": "steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": hs["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": ("f64" if head.startswith("fp64") else
                      "f64 products as bf16 slices (Ozaki) / tf32x3 search / f64 factorisations"),
            "data": "synthetic (seeded shear-jet initial condition)",
            "timing": ("CUDA events on the stepping stream" if B == 1 else
                       "host clock between device-wide synchronisations (library-owned streams)"),
            "config": {**w, "precision": head, "parallelism": f"replicas x{world}",
                       "trajectories": B, "stage_graphs": bool(graphs),
                       "step_graphs": graphs == 2,
                       "stage_graph_replays_timed": hs["step_graph_replays_timed"],
                       "l2": "flushed between timed steps (256 MB write)",
                       "all_projections_converged": hs["all_projections_converged"]},
            "e2e": e2e, "gpu_launches": hs["gpu_launches"], "roofline": hs["roofline"],
            "tc_subspace_searches_timed": hs["tc_subspace_searches_timed"],
            "cpu_baseline": cpu, "clocks": clocks, "wall_s": hs["wall_s"]}
    implicit_form = ("the paper's implicit right-hand side (nonlinear terms inside the "
                     "projection's environments)")
    if head == "mixed_implicit":
        line["form"] = implicit_form + ", mixed precision"
        line["fp64_implicit"] = sums["fp64_implicit"]
        line["fp64_implicit"]["form"] = implicit_form + ", FP64"
        line["mixed_vs_fp64_rel_l2"] = cmp_mi
        line["mixed_vs_fp64_forms"] = ["mixed_implicit", "fp64_implicit"]
        line["mixed_vs_fp64_after_steps"] = steps_taken
        line["mixed_over_fp64"] = hs["value"] / sums["fp64_implicit"]["value"]
        if "mixed" in names:
            line["mixed_explicit"] = sums["mixed"]
            line["mixed_explicit"]["form"] = "explicit right-hand side (B formed), mixed precision"
            line["mixed_explicit_vs_fp64_rel_l2"] = cmp
        if "fp64" in names:
            line["fp64"] = sums["fp64"]
            line["fp64"]["form"] = "explicit right-hand side (B formed), FP64"
            line["fp64_implicit_vs_fp64_rel_l2"] = cmp_imp
            line["mixed_over_fp64_explicit"] = hs["value"] / sums["fp64"]["value"]
    elif "mixed" in names and "fp64" in names:
        line["fp64"] = sums["fp64"]
        line["mixed_vs_fp64_rel_l2"] = cmp
        line["mixed_vs_fp64_after_steps"] = steps_taken
        line["mixed_over_fp64"] = hs["value"] / sums["fp64"]["value"]
    if tcg:
        line["tc_gemm"] = tcg
    if ozg:
        line["oz_gemm"] = ozg
    line["peaks_file"] = {k: peaks.get(k) for k in ("hbm_gbs", "bf16_tflops")}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    if len(sys.argv) == 3 and sys.argv[1] == "--oracle-steps":
        _oracle_steps_child(sys.argv[2])
        sys.exit(0)
    sys.exit(main())
