"""The bench's N > 1 path on the CPU: world-size-2 gloo process groups (no GPU).

bench.py runs one replica of the workload per GPU ("replicas only": the single
grid has no shard without an exchange step, and the runs here have one GPU).
What is host logic - the max-over-ranks time, the whole-job throughput, the
reference arm's rank-0-only output - runs here with the gloo backend.
"""

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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, _ = bench.dist_env()
        t = bench.max_over_ranks(torch, 10.0 + 5.0 * rank, torch.device("cpu"))  # rank 1 is the slow one
        out[rank] = (w, r, t, bench.job_gflops(w, 2.0e9, t))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_throughput_gloo():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        w, r, t, v = res[rank]
        assert (w, r) == (world, rank)
        assert t == 15.0  # every rank sees the slowest rank's time
        assert abs(v - world * 2.0e9 / 15e-3 / 1e9) < 1e-9


def test_single_process_aggregation_is_identity():
    import bench
    assert bench.max_over_ranks(torch, 3.5, torch.device("cpu")) == 3.5
    assert bench.job_gflops(1, 1.0e9, 1.0) == 1000.0


@pytest.mark.slow
def test_reference_arm_under_torchrun_prints_once():
    """--impl reference with two ranks: rank 0 times the oracle and prints one JSON line, rank 1 exits 0."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "3", "--reference-budget-s", "4"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
