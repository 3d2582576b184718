"""The multi-rank host logic of bench.py on CPU (gloo, world size 2).

bench.py runs one replica per GPU under torchrun and reports the whole-job
throughput from the MAXIMUM of the ranks' timed regions; the reference arm
runs on rank 0 only and the other ranks exit without work.  Both are
checked here without a GPU.
"""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.reduce_max_time(1.0 + 0.5 * rank, dist, "cpu")
    q.put((rank, t))
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_max_time_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert got == {0: 1.5, 1: 1.5}


def test_reduce_max_time_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max_time(0.25) == 0.25


def test_reference_arm_prints_once_under_torchrun():
    port = free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl",
           "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--grid-bits", "3"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600,
                       env=dict(os.environ, CUDA_VISIBLE_DEVICES=""))
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(l) for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = lines[0]
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["config"]["n"] == 3 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["steps"] == 1 and line["algorithmic_flops_per_step"] > 0
    # the timed region really holds steps x ms_per_step of oracle work
    assert line["ms_per_step"] > 0


def test_flop_counter_models():
    """The oracle's FLOP counter: products 2 x output x contracted size,
    Householder QR with explicit Q 4mn^2 - 4n^3/3, thin SVD 6mn^2 + 20n^3."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    c = bench.FlopCounter().install()
    try:
        a, b = np.ones((3, 4, 2)), np.ones((4, 2, 5))
        np.tensordot(a, b, ([1, 2], [0, 1]))
        assert c.total == 2 * 3 * 5 * 8
        c.total = 0.0
        np.einsum("ab,bc->ac", np.ones((3, 4)), np.ones((4, 5)))
        assert c.total == 2 * 3 * 4 * 5
        c.total = 0.0
        np.linalg.qr(np.ones((6, 4)))
        assert abs(c.total - (4 * 6 * 16 - 4 / 3 * 64)) < 1e-9
        c.total = 0.0
        np.linalg.svd(np.eye(4, 7), full_matrices=False)
        assert c.total == 6 * 7 * 16 + 20 * 64
    finally:
        c.uninstall()
    c.total = 0.0
    np.tensordot(np.ones((2, 2)), np.ones((2, 2)), 1)
    assert c.total == 0.0
