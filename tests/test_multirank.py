"""Multi-GPU host logic on CPU (world size 2, gloo): the path shards by screen with no
data-path collective, so what needs checking is that ranks get disjoint workloads of the
same shape, that the job's step time is the slowest rank's, and that the reference arm
prints one line from rank 0 under torchrun."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_rank_workloads_are_disjoint_and_alike():
    for name in ("batched", "profile", "single4096"):
        a, _ = bench._workload(name, 0)
        b, _ = bench._workload(name, 1)
        assert [x["n"] for x in a] == [x["n"] for x in b]
        assert {x["seed"] for x in a}.isdisjoint({x["seed"] for x in b})
        for x, y in zip(a, b):
            np.testing.assert_array_equal(x["lambdas_nm"], y["lambdas_nm"])


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench._max_over_ranks(10.0 + 5.0 * rank, world, "cpu")
    q.put((rank, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_step_time_is_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29000 + os.getpid() % 2000
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = dict(q.get(timeout=10) for _ in range(2))
    assert got == {0: 15.0, 1: 15.0}
    assert bench._max_over_ranks(7.5, 1, "cpu") == 7.5


def test_reference_arm_prints_once_under_torchrun():
    port = 31000 + os.getpid() % 2000
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
