"""The N > 1 path on CPU (gloo, world_size 2): replicas with no data-path
collective.  The whole-job aggregation takes the slowest rank's time and the sum of
the ranks' zone-updates; each rank draws its own batch (seed + rank); under
torchrun the reference arm prints one line, from rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, z = bench.aggregate_over_ranks(1.0 + rank, 100.0 * (rank + 1), world)
    from paper_2212_00370_gb300 import workloads as W
    w = W.riemann_batch(8, seed=W.SEED_BASE + 1 + rank, nmin=16, nmax=32)
    q.put((rank, t, z, float(w.V[0].sum())))
    dist.destroy_process_group()


def test_aggregate_over_two_gloo_ranks():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, z, _ in res:
        assert t == 2.0 and z == 300.0          # max time, summed work, on every rank
    assert res[0][3] != res[1][3]               # each rank its own problems


def test_reference_arm_under_torchrun_prints_one_line():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "1", "--instances", "32", "--cpu-sample", "16"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    out = json.loads(lines[0])
    assert out["impl"] == "reference" and out["value"] > 0 and out["unit"] == "zone-updates/s"
    assert out["e2e"]["h2d_bytes_per_step"] == 0 and out["cpu_baseline"]["kind"] == "oracle"
