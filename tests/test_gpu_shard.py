"""Walker sharding on the GPU: contexts that each hold one shard of every
group (``shard=(rank, count)``), merged after every iteration, against one
context holding all the walkers and against the oracle.

Two shards run side by side in one process on one GPU (their kernels do not
wait on each other); the merge sums their histograms on the host.  The
sharded merge helper is also run as a one-rank process group, with NCCL on
device tensors and gloo on host tensors.
"""
import os
import socket

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

GROUPS = [{"L": 8, "T": 1.4182, "n_walkers": 37}, {"L": 12, "T": 0.9, "n_walkers": 20},
          {"L": 48, "T": 0.9, "n_walkers": 9}]
SEED, N_ITER, SWEEPS, N_MEAS = 7, 3, 12, 5


def muca():
    from paper_1502_07214_gb300 import muca as m

    return m


def run_unsharded():
    c = muca().Context(GROUPS, seed=SEED)
    hists = []
    for _ in range(N_ITER):
        c.sweep_iter(SWEEPS)
        hists.append([c.get_hist(g) for g in range(len(GROUPS))])
        c.merge_update()
    c.reserve_timeseries(N_MEAS)
    c.sweep_iter(N_MEAS, record=True)
    res = [(c.get_state(g), c.get_lnW(g), c.get_timeseries(g)) for g in range(len(GROUPS))]
    c.close()
    return hists, res


def test_two_shards_equal_one_context():
    """Shards 0 and 1 of 2 (walkers [0, W/2) and [W/2, W) of every group):
    the summed histograms of every iteration, the weights, the walkers'
    spins and tallies and the recorded series (shards side by side on the
    walker axis) equal the unsharded context's, bit for bit."""
    want_h, want = run_unsharded()
    ctx = [muca().Context(GROUPS, seed=SEED, shard=(r, 2)) for r in range(2)]
    for g, spec in enumerate(GROUPS):
        n0, n1 = ctx[0].specs[g]["n_walkers"], ctx[1].specs[g]["n_walkers"]
        assert n0 + n1 == spec["n_walkers"] and n0 == spec["n_walkers"] // 2
        assert ctx[1].specs[g]["first_walker"] == ctx[0].specs[g]["first_walker"] + n0
    for it in range(N_ITER):
        for c in ctx:
            c.sweep_iter(SWEEPS)
        for g in range(len(GROUPS)):
            H = ctx[0].get_hist(g) + ctx[1].get_hist(g)
            assert np.array_equal(H, want_h[it][g]), (it, g)
            for c in ctx:
                c.set_hist(g, H)
        for c in ctx:
            c.merge_update()
    for c in ctx:
        c.reserve_timeseries(N_MEAS)
        c.sweep_iter(N_MEAS, record=True)
    for g in range(len(GROUPS)):
        (spins, tal), lnW, ts = want[g]
        parts = [(c.get_state(g), c.get_lnW(g), c.get_timeseries(g)) for c in ctx]
        assert np.array_equal(np.concatenate([p[0][0] for p in parts]), spins), g
        assert np.array_equal(np.concatenate([p[0][1] for p in parts]), tal), g
        for p in parts:
            assert np.array_equal(p[1], lnW), g
        assert np.array_equal(np.concatenate([p[2] for p in parts], axis=2), ts), g
    for c in ctx:
        c.close()


def test_shard_against_the_oracle():
    """Shard 2 of 3 of the L = 8 group follows the oracle's walkers with the
    same global ids under the oracle's weights of the whole group."""
    L, T, W = 8, 1.4182, 37
    ref = oracle.muca_run(L, T, W, SEED, N_ITER, SWEEPS)
    c = [muca().Context([{"L": L, "T": T, "n_walkers": W}], seed=SEED, shard=(r, 3))
         for r in range(3)]
    for _ in range(N_ITER):
        for x in c:
            x.sweep_iter(SWEEPS)
        H = sum(x.get_hist(0) for x in c)
        for x in c:
            x.set_hist(0, H)
            x.merge_update()
    lo = c[2].specs[0]["first_walker"]
    spins, tal = c[2].get_state(0)
    assert lo == W * 2 // 3
    assert np.array_equal(spins, ref["spins"][lo:])
    assert np.array_equal(tal, ref["tallies"][lo:])
    assert np.array_equal(c[2].get_lnW(0), ref["lnW"])
    for x in c:
        x.close()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("backend,device", [("nccl", True), ("gloo", False)])
def test_sharded_merge_helper_one_rank(backend, device):
    """The product's sharded merge (shard.merge_update) in a one-rank process
    group, device all-reduce with NCCL or host all-reduce with gloo: a run
    through it equals the unsharded run."""
    import torch.distributed as dist

    from paper_1502_07214_gb300 import shard

    want_h, want = run_unsharded()
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_free_port()))
    kw = {"device_id": torch.device("cuda", 0)} if backend == "nccl" else {}
    dist.init_process_group(backend, rank=0, world_size=1, **kw)
    try:
        c = muca().Context(GROUPS, seed=SEED, shard=(0, 1))
        for _ in range(N_ITER):
            c.sweep_iter(SWEEPS)
            shard.merge_update(c, dist.all_reduce, device=device)
        for g in range(len(GROUPS)):
            assert np.array_equal(c.get_lnW(g), want[g][1]), g
        c.reserve_timeseries(N_MEAS)
        c.sweep_iter(N_MEAS, record=True)
        for g in range(len(GROUPS)):
            (spins, tal), _, ts = want[g]
            assert np.array_equal(c.get_state(g)[0], spins), g
            assert np.array_equal(c.get_state(g)[1], tal), g
            assert np.array_equal(c.get_timeseries(g), ts), g
        c.close()
    finally:
        dist.destroy_process_group()


def test_shard_checkpoint_is_bound_to_its_shard(tmp_path):
    """A checkpoint records its shard: it restores into the same shard (and
    the run continues bit-identically), not into another one."""
    path = str(tmp_path / "shard.ck")
    a = muca().Context(GROUPS[:1], seed=SEED, shard=(1, 2))
    a.sweep_iter(5)
    a.checkpoint(path)
    a.sweep_iter(4)
    sa = a.get_state(0)[0]
    a.close()
    b = muca().Context(GROUPS[:1], seed=SEED, shard=(1, 2))
    b.restore(path)
    b.sweep_iter(4)
    assert np.array_equal(b.get_state(0)[0], sa)
    b.close()
    c = muca().Context(GROUPS[:1], seed=SEED, shard=(0, 2))
    with pytest.raises(muca().MucaError) as e:
        c.restore(path)
    assert e.value.code == muca().ERR_INVALID_ARG
    c.close()
    with pytest.raises(muca().MucaError):
        muca().Context([{"L": 4, "T": 1.0, "n_walkers": 2}], shard=(0, 3))
