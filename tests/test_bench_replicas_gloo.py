"""The multi-GPU bench path on CPU: two gloo ranks, each with its own replica
time and atom count; the whole-job value is the atoms of all ranks over the
slowest rank's time (replicas only, no data-path collective)."""
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        value, ms = bench.job_throughput(10.0 + rank, 1000.0 * (rank + 1), 5, dist, "cpu")
        if rank == 0:
            with open(out, "w") as f:
                json.dump({"value": value, "ms": ms}, f)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    out = str(tmp_path / "r0.json")
    mp.start_processes(_rank, args=(2, _free_port(), out), nprocs=2, join=True,
                       start_method="spawn")
    r = json.load(open(out))
    assert r["ms"] == 11.0
    assert r["value"] == pytest.approx(3000.0 * 5 / 0.011, rel=1e-12)


def test_single_rank_is_local():
    sys.path.insert(0, ROOT)
    import bench
    v, ms = bench.job_throughput(4.0, 1000.0, 10)
    assert ms == 4.0 and v == pytest.approx(1000.0 * 10 / 0.004)
