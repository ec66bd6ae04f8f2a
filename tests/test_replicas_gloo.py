"""The multi-GPU path is replicas only: each rank runs the whole workload on
its own GPU, the job's time is the slowest rank's and its throughput the sum.
These world-size-2 tests run that host logic with the gloo backend on CPU."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r takes 0.1 (r + 1) s for the same 5 units of work: the job takes
        # the slowest rank's 0.2 s and does world x 5 units
        t = bench.max_over_ranks(0.1 * (rank + 1), dist)
        rate, t_max = bench.replica_throughput(5.0, 0.1 * (rank + 1), world, dist)
        out[rank] = (t, rate, t_max)
    finally:
        dist.destroy_process_group()


def test_replica_aggregation_world_size_two():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        t, rate, t_max = res[r]
        assert t == pytest.approx(0.2) and t_max == pytest.approx(0.2)
        assert rate == pytest.approx(world * 5.0 / 0.2)      # 10 units in the slowest rank's 0.2 s


def test_single_process_needs_no_backend():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(0.3) == 0.3
    assert bench.replica_throughput(6.0, 0.5, 1) == (12.0, 0.5)


@pytest.mark.slow
def test_reference_arm_under_torchrun_prints_once():
    # two ranks: rank 0 times the oracle and prints one JSON line, rank 1 exits 0
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", "--master-port=%d" % port, os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
