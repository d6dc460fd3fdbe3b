"""The benchmark's N > 1 path on CPU: world-size-2 gloo ranks, replicas only.

Each rank runs an independent replica; the job's value is all ranks' units over
the slowest rank's time.  Here two gloo ranks feed different local times through
bench.aggregate_replicas and must agree on the maximum and the job value.
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    total, value = bench.aggregate_replicas(torch, world, 1.0 + rank, 1000, torch.device("cpu"))
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, total, value))


def test_replica_aggregation_over_two_gloo_ranks():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, total, value in out:
        assert total == 2.0                  # the slower rank's time
        assert value == 2 * 1000 / 2.0       # both ranks' units over it


def test_single_rank_aggregation_is_local():
    import torch
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_replicas(torch, 1, 4.0, 100, torch.device("cpu")) == (4.0, 25.0)


def test_reference_arm_prints_one_line_from_the_oracle():
    """bench.py --impl reference times the FP64 oracle on the host cores on a
    bounded sample of the workload and prints one JSON line."""
    import json
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--cpu-seconds", "1"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "particle-steps/s"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
