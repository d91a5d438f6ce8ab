"""Walker sharding over processes (one GPU each): the merge step of the
parallel multicanonical scheme (Sec. II) across shards.

Within one iteration the walkers are independent given the weights, so a
group's walkers can be split over N contexts (``Context(..., shard=(rank,
N))``), each sweeping its own walkers with the global walker ids of the
unsharded run.  The merge then sums the shards' integer histograms (one
all-reduce per group and iteration; integer sums do not depend on the order
of the ranks) and every rank runs the same deterministic FP64 weight update
and table build on the same merged histogram, so every rank holds the same
weights and tables, bit for bit, as one context holding all the walkers.

The all-reduce is the caller's: any callable that sums a torch int64 tensor
in place over the ranks, e.g. ``torch.distributed.all_reduce`` with NCCL on
device tensors or gloo on CPU tensors.
"""
import numpy as np

from . import muca


def merge_update(ctx, all_reduce, device=True):
    """One sharded merge and weight update of every group of ctx: each
    group's histogram is summed over the ranks by ``all_reduce`` (on a CUDA
    tensor if device, else on a CPU tensor), written back, and
    ``muca_merge_update`` runs on the merged histograms."""
    import torch

    for g in range(len(ctx.specs)):
        n_e = ctx.n_e(g)
        if device:
            t = torch.empty(n_e, dtype=torch.int64, device="cuda")
            ctx.get_hist_device(g, t)
            all_reduce(t)
            torch.cuda.current_stream().synchronize()
            ctx.set_hist_device(g, t)
        else:
            t = torch.from_numpy(ctx.get_hist(g).astype(np.int64))
            all_reduce(t)
            ctx.set_hist(g, t.numpy().astype(np.uint64))
    ctx.merge_update()


def host_merge_update(hist_local, lnW, all_reduce, kind=muca.REC_PLAIN, acc=None):
    """The host part of a sharded merge without a context: sum this rank's
    histogram (uint64 [n_e]) over the ranks and apply the library's host FP64
    weight update (``muca_weight_update``) to lnW (and acc) in place.
    Returns the merged histogram."""
    import torch

    t = torch.from_numpy(np.ascontiguousarray(hist_local, dtype=np.uint64).astype(np.int64))
    all_reduce(t)
    merged = t.numpy().astype(np.uint64)
    muca.weight_update(kind, merged, lnW, acc)
    return merged


def walker_range(ctx, g, all_reduce_max):
    """(min, max) of the current E_Delta over the walkers of group g on every
    rank: the window that an adaptive run (``Context.set_window``) starts from
    must be the same on every shard.  ``all_reduce_max`` takes the maximum of
    a CPU int64 tensor in place over the ranks."""
    import torch

    lo, hi = ctx.walker_range(g)
    t = torch.tensor([-lo, hi], dtype=torch.int64)
    all_reduce_max(t)
    return -int(t[0]), int(t[1])


def shard_range(n_walkers, rank, count):
    """Walkers [lo, hi) of a group of n_walkers held by shard rank of count
    (the rule of ``muca_options.shard_rank / shard_count``)."""
    if count <= 1:
        return 0, n_walkers
    return n_walkers * rank // count, n_walkers * (rank + 1) // count
