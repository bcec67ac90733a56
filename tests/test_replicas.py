"""Multi-GPU path of the bench: replicas with no collective on the data path,
max-over-ranks timing - exercised with world_size 2 on CPU (gloo)."""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        total = [12.5, 20.0][rank]             # rank 1 is the slowest
        m = bench.max_over_ranks(total, torch.device("cpu"))
        out[rank] = (m, bench.replica_events_per_s(world, 100, m))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_throughput_with_two_gloo_ranks():
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    out = mp.get_context("spawn").Manager().dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    for r in range(2):
        m, v = out[r]
        assert m == 20.0                       # every rank reports the slowest rank's time
        assert v == pytest.approx(2 * 100 / 0.020)


def test_single_process_is_unchanged():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.0, torch.device("cpu")) == 3.0
    assert bench.replica_events_per_s(1, 10, 5.0) == pytest.approx(2000.0)
