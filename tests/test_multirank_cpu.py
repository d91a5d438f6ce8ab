"""The N-GPU form of the benchmark runs one independent replica per rank and
reports the whole job's rate over the slowest rank.  Its cross-rank steps run
here as two gloo ranks on the CPU (no GPU involved)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys

    sys.path.insert(0, os.path.dirname(HERE))
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r times 10 (r + 1) ms for 1000 units
        rate, ms = bench.job_rate(10.0 * (rank + 1), 1000, world, dist)
        out[rank] = (rate, ms, bench.replica_seed(3, rank))
    finally:
        dist.destroy_process_group()


def test_two_ranks_rate_over_the_slowest_rank():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        rate, ms, seed = res[r]
        assert ms == 20.0  # the slower rank's time, on every rank
        assert rate == pytest.approx(2 * 1000 / 0.020)
    assert res[0][2] != res[1][2]  # independent replicas


def test_one_rank_needs_no_process_group():
    import sys

    sys.path.insert(0, os.path.dirname(HERE))
    import bench

    rate, ms = bench.job_rate(12.5, 500, 1)
    assert ms == 12.5 and rate == pytest.approx(500 / 0.0125)
