"""The N-GPU form of the benchmark and the walker-sharded merge (Sec. II's
parallel scheme over ranks).  Their cross-rank steps run here as two gloo
ranks on the CPU (no GPU involved): the whole job's rate over the slowest
rank, a sharded run whose merged histograms, weights and tables equal one
rank holding all the walkers, and a rank that leaves between iterations
(the next merge ends with an error instead of hanging, and the weights stay
those of the last good merge)."""
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
        out[rank] = (rate, ms, bench.shard_group(48, 0.9, 4096, world)["n_walkers"])
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
    assert res[0][2] == res[1][2] == 2 * 4096  # one simulation of both ranks' walkers


def test_one_rank_needs_no_process_group():
    import sys

    sys.path.insert(0, os.path.dirname(HERE))
    import bench

    rate, ms = bench.job_rate(12.5, 500, 1)
    assert ms == 12.5 and rate == pytest.approx(500 / 0.0125)


def _shard_rank(rank, world, port, out):
    """One rank of a sharded run: the oracle sweeps this rank's walkers (the
    test's stand-in for a GPU), the product's sharded host merge sums the
    histograms over the ranks and updates lnW, and the product's host table
    build gives the next iteration's table."""
    import sys

    sys.path.insert(0, os.path.dirname(HERE))
    import numpy as np

    import oracle
    from paper_1502_07214_gb300 import muca, shard

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        L, T, W, seed, n_iter, sweeps = SHARD_RUN
        V = L ** 3
        lo, hi = shard.shard_range(W, rank, world)
        spins = {w: oracle.init_spins(L, seed, w) for w in range(lo, hi)}
        tal = {w: oracle.energies(L, spins[w]).astype(np.int32) for w in spins}
        lnW = np.zeros(V + 1)
        table = muca.build_table(L, T, 0, V, lnW)
        merged = []
        for it in range(n_iter):
            H = np.zeros(V + 1, dtype=np.uint64)
            for w in spins:
                oracle.sweeps(L, 0, V, table, seed, w, it * sweeps, sweeps, spins[w], tal[w],
                              hist=H)
            merged.append(shard.host_merge_update(H, lnW, dist.all_reduce))
            table = muca.build_table(L, T, 0, V, lnW)
        out[rank] = (np.array(merged), lnW, table, {w: spins[w] for w in spins})
    finally:
        dist.destroy_process_group()


# L, T, walkers, seed, iterations, sweeps per iteration of the sharded run
SHARD_RUN = (4, 1.0, 13, 5, 4, 30)


def test_two_ranks_sharded_merge_equals_one_rank():
    """Walkers sharded over two gloo ranks (6 and 7 of 13): after every
    iteration the all-reduced histogram equals the merged histogram of one
    oracle run holding all the walkers, and the weights, the tables and every
    walker's spins are bit-identical to that run."""
    import sys

    sys.path.insert(0, os.path.dirname(HERE))
    import numpy as np

    import oracle

    L, T, W, seed, n_iter, sweeps = SHARD_RUN
    V = L ** 3
    ref = oracle.muca_run(L, T, W, seed, n_iter, sweeps)
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_shard_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        merged, lnW, table, spins = res[r]
        assert np.array_equal(merged, ref["hist"]), r
        assert np.array_equal(lnW, ref["lnW"]), r
        assert np.array_equal(table, oracle.build_table(L, T, 0, V, ref["lnW"])), r
        for w, s in spins.items():
            assert np.array_equal(s, ref["spins"][w]), (r, w)
    assert sorted(w for r in range(world) for w in res[r][3]) == list(range(W))


def _leaving_rank(rank, world, port, out, stall=0.0):
    """Rank 1 takes part in the first merge, then leaves between iterations:
    its process ends without joining the second merge, after `stall` seconds
    alive (a rank that hangs); rank 0 runs its second merge with a short
    process-group timeout."""
    import sys
    from datetime import timedelta

    sys.path.insert(0, os.path.dirname(HERE))
    import time

    import numpy as np

    from paper_1502_07214_gb300 import muca, shard

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=timedelta(seconds=5))
    V = 64
    lnW = np.zeros(V + 1)
    H = np.full(V + 1, 3 + rank, dtype=np.uint64)
    merged = shard.host_merge_update(H, lnW, dist.all_reduce)
    if rank == 1:
        out[rank] = ("left", merged.copy(), lnW.copy())
        time.sleep(stall)
        return  # leaves between iterations: no destroy, no second merge
    before = lnW.copy()
    t0 = time.monotonic()
    try:
        shard.host_merge_update(H, lnW, dist.all_reduce)
        outcome = "merged"
    except Exception as e:  # the missing rank ends the collective with an error
        outcome = type(e).__name__
    waited = time.monotonic() - t0
    # the library still serves this rank: a local update on a copy of the weights
    probe = lnW.copy()
    muca.weight_update(muca.REC_PLAIN, H, probe)
    out[rank] = (outcome, merged.copy(), lnW.copy(), before, waited, probe)
    try:
        dist.destroy_process_group()
    except Exception:
        pass


@pytest.mark.parametrize("stall", [0.0, 12.0])
def test_a_rank_that_leaves_ends_the_next_merge_with_an_error(stall):
    """Failure detection on the host: after one good merge (both ranks' integer
    histograms summed), rank 1 leaves between iterations, at once (its
    connections close) or after hanging for longer than the process group's
    5 s timeout.  Rank 0's next merge does not hang: the collective ends with
    an error (at once, or when the timeout runs out), and rank 0's weights are
    those of the last good merge (the update runs only on a merged
    histogram), so the run can continue from its last checkpoint."""
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_leaving_rank, args=(world, port, out, stall), nprocs=world, join=True)
        res = dict(out)
    import numpy as np

    outcome, merged0, lnW0, before, waited, probe = res[0]
    left, merged1, lnW1 = res[1]
    assert left == "left"
    assert np.array_equal(merged0, np.full(65, 7, dtype=np.uint64))
    assert np.array_equal(merged0, merged1) and np.array_equal(lnW1, before)
    assert np.allclose(before, -np.log(7.0))  # lnW -= ln H after the good merge
    assert outcome != "merged", "a merge without rank 1 must not succeed"
    assert np.array_equal(lnW0, before), "a failed merge must leave lnW unchanged"
    assert waited < (2.0 if stall == 0.0 else 11.0)
    assert np.allclose(probe, before - np.log(3.0))
