"""Multi-GPU runs are replicas (independent simulations need no exchange): the host logic
that shards simulations over ranks and forms the whole-job numbers, on world_size 2 with
the gloo backend on the CPU, and the reference arm under torchrun (rank 0 alone prints)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = bench.shard(10, rank, world)
    pushes, secs = bench.job_totals(100.0 * (rank + 1), 0.5 + rank, world)
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    q.put((rank, mine, pushes, secs, gathered))
    dist.destroy_process_group()


def test_shards_and_whole_job_totals_on_two_gloo_ranks():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mine, pushes, secs, gathered in out:
        assert pushes == 300.0          # sum over ranks
        assert secs == 1.5              # slowest rank
        flat = sorted(i for g in gathered for i in g)
        assert flat == list(range(10))  # every simulation once
        assert set(gathered[0]).isdisjoint(gathered[1])


def test_reference_arm_prints_once_under_torchrun():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--workload", "1d", "--steps", "2", "--warmup", "1", "--gpus", "2"]
    r = subprocess.run(cmd, capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
