"""The adaptive E_Delta window (the reading of the weight iteration's window
that the oracle states as R15) on the GPU, against the oracle, bit for bit.

Every group starts in the range of its walkers' initial E_Delta and grows by
its step after every iteration whose histogram is flat over the window; the
per-iteration histograms and windows, the final weights, spins, tallies and
the measurement series equal the oracle's, in the plain and the graph form,
with both weight recursions and in every kernel kind.
"""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

SEED, N_ITER, N_MEAS = 21, 60, 12
# (group, grow_flat, grow_step, sweeps): growth at every size that grows
# within N_ITER iterations (L = 4, 8, 3) and one whose window stays (L = 12
# at T = 0.9, inside the first-order regime)
GROUPS = [({"L": 4, "T": 1.0, "n_walkers": 40}, 0.5, 4),
          ({"L": 8, "T": 1.4182, "n_walkers": 24}, 0.2, 8),
          ({"L": 12, "T": 0.9, "n_walkers": 20}, 0.2, 12),
          ({"L": 3, "T": 2.0, "n_walkers": 33}, 0.5, 2)]
SWEEPS = 100


def muca():
    from paper_1502_07214_gb300 import muca as m

    return m


def oracle_runs(groups, recursion, n_iter=N_ITER, n_meas=N_MEAS):
    """The oracle's run of every group (walker ids continue across groups, as
    in one context); returns the runs and each group's initial window."""
    out, wins, id0 = [], [], 0
    for spec, flat, step in groups:
        L, W = spec["L"], spec["n_walkers"]
        e = [int(oracle.energies(L, oracle.init_spins(L, SEED, id0 + w))[1]) for w in range(W)]
        win0 = (min(e), max(e))
        out.append(oracle.muca_run(L, spec["T"], W, SEED, n_iter, SWEEPS, n_meas=n_meas,
                                   walker_id0=id0, window=win0, grow_flat=flat, grow_step=step,
                                   recursion=recursion))
        wins.append(win0)
        id0 += W
    return out, wins


def gpu_context(groups, recursion, **kw):
    c = muca().Context([g for g, _, _ in groups], seed=SEED, **kw)
    c.set_recursion(recursion)
    for i, (_, flat, step) in enumerate(groups):
        lo, hi = c.walker_range(i)
        c.set_window(i, lo, hi, flat, step)
    return c


def check_final(c, refs, n_groups):
    for i in range(n_groups):
        ref = refs[i]
        spins, tal = c.get_state(i)
        assert np.array_equal(c.get_lnW(i), ref["lnW"]), i
        assert np.array_equal(spins, ref["spins"]), i
        assert np.array_equal(tal, ref["tallies"]), i
        assert c.get_window(i) == tuple(int(x) for x in ref["windows"][-1]), i
        assert np.array_equal(c.get_timeseries(i), ref["ts"].transpose(1, 2, 0)), i


@pytest.mark.parametrize("recursion", [0, 1])
def test_plain_form_every_iteration(recursion):
    """Kernel configuration chosen by the autotuner; after every iteration the
    merged histogram and the new window equal the oracle's."""
    refs, wins = oracle_runs(GROUPS, recursion)
    c = gpu_context(GROUPS, recursion)
    for i in range(len(GROUPS)):
        assert c.get_window(i) == wins[i]
    grew = [0] * len(GROUPS)
    for it in range(N_ITER):
        c.sweep_iter(SWEEPS)
        hists = [c.get_hist(i) for i in range(len(GROUPS))]
        c.merge_update()
        for i in range(len(GROUPS)):
            assert np.array_equal(hists[i], refs[i]["hist"][it]), (it, i)
            w = c.get_window(i)
            assert w == tuple(int(x) for x in refs[i]["windows"][it]), (it, i)
            grew[i] += w != (tuple(refs[i]["windows"][it - 1]) if it else wins[i])
    c.reserve_timeseries(N_MEAS)
    c.sweep_iter(N_MEAS, record=True)
    check_final(c, refs, len(GROUPS))
    assert grew[0] >= 3 and grew[1] >= 3 and grew[3] >= 3, grew
    c.close()


@pytest.mark.parametrize("recursion", [0, 1])
@pytest.mark.parametrize("residency,wpb,P", [(0, 0, 0), (1, 8, 4), (2, 16, 1), (3, 32, 0),
                                             (4, 0, 0)])
def test_graph_form_in_every_kernel_kind(recursion, residency, wpb, P):
    """The whole weight iteration as one CUDA graph (the growth runs in its
    host node) in each kernel kind, forced; row lengths 4, 8, 12 (the
    split kind runs L = 8, 12 and leaves L = 4 to the global kind; the
    row-scan kind fixes its own walkers and lanes per row length)."""
    groups = GROUPS[:3]
    refs, _ = oracle_runs(groups, recursion)
    kw = {} if residency == 0 else {"residency": residency, "walkers_per_block": wpb,
                                     "lanes_per_walker": P}
    c = gpu_context(groups, recursion, **kw)
    for i, (spec, _, _) in enumerate(groups):
        # the split kind takes 8 <= L <= 48; L = 4 falls back to the global kind
        want = residency if residency != 3 or spec["L"] >= 8 else 1
        assert residency == 0 or c.get_config(i)[0] == want, (i, c.get_config(i))
    c.run_graph(N_ITER, SWEEPS)
    c.reserve_timeseries(N_MEAS)
    c.sweep_iter(N_MEAS, record=True)
    check_final(c, refs, len(groups))
    c.close()


def test_iterate_stops_once_the_full_window_is_flat():
    """muca_iterate stops after the first iteration whose histogram was taken
    over the whole [0, V] and is flat; the oracle's histograms and windows give
    that iteration."""
    groups = [GROUPS[3]]
    refs, wins = oracle_runs(groups, 0, n_iter=N_ITER, n_meas=0)
    ref = refs[0]
    V = groups[0][0]["L"] ** 3
    ran = [wins[0]] + [tuple(int(x) for x in w) for w in ref["windows"][:-1]]
    want = None
    for it in range(N_ITER):
        lo, hi = ran[it]
        if (lo, hi) == (0, V) and oracle.flatness(ref["hist"][it])[0] >= 0.6:
            want = it + 1
            break
    assert want is not None and want > 1
    c = gpu_context(groups, 0)
    n = c.iterate(N_ITER, SWEEPS, 0.6)
    assert n == want
    ref = oracle.muca_run(3, 2.0, 33, SEED, n, SWEEPS, window=wins[0], grow_flat=0.5, grow_step=2)
    assert np.array_equal(c.get_lnW(0), ref["lnW"])
    assert np.array_equal(c.get_state(0)[0], ref["spins"])
    c.close()


def test_checkpoint_carries_the_window(tmp_path):
    """A checkpoint taken while the window is still growing restores it with
    its rule: the continued run equals the uninterrupted one."""
    groups = GROUPS[:2]
    path = str(tmp_path / "win.ck")
    a = gpu_context(groups, 1)
    for _ in range(20):
        a.sweep_iter(SWEEPS)
        a.merge_update()
    a.checkpoint(path)
    wa = [a.get_window(i) for i in range(2)]
    for _ in range(20):
        a.sweep_iter(SWEEPS)
        a.merge_update()
    b = muca().Context([g for g, _, _ in groups], seed=SEED)
    b.restore(path)
    assert [b.get_window(i) for i in range(2)] == wa
    for _ in range(20):
        b.sweep_iter(SWEEPS)
        b.merge_update()
    for i in range(2):
        assert b.get_window(i) == a.get_window(i)
        assert np.array_equal(b.get_lnW(i), a.get_lnW(i))
        assert np.array_equal(b.get_state(i)[0], a.get_state(i)[0])
    a.close()
    b.close()


def test_two_shards_share_one_window():
    """Two walker shards that start from the window of all the walkers and
    merge their histograms equal the oracle's run of the whole group."""
    spec, flat, step = GROUPS[1]
    refs, wins = oracle_runs([GROUPS[1]], 0, n_iter=30, n_meas=0)
    ctx = [muca().Context([spec], seed=SEED, shard=(r, 2)) for r in range(2)]
    ranges = [c.walker_range(0) for c in ctx]
    lo, hi = min(r[0] for r in ranges), max(r[1] for r in ranges)
    assert (lo, hi) == wins[0]
    for c in ctx:
        c.set_window(0, lo, hi, flat, step)
    for it in range(30):
        for c in ctx:
            c.sweep_iter(SWEEPS)
        H = ctx[0].get_hist(0) + ctx[1].get_hist(0)
        assert np.array_equal(H, refs[0]["hist"][it]), it
        for c in ctx:
            c.set_hist(0, H)
            c.merge_update()
            assert c.get_window(0) == tuple(int(x) for x in refs[0]["windows"][it]), it
    n0 = ctx[0].specs[0]["n_walkers"]
    for r, c in enumerate(ctx):
        assert np.array_equal(c.get_lnW(0), refs[0]["lnW"])
        sl = slice(0, n0) if r == 0 else slice(n0, None)
        assert np.array_equal(c.get_state(0)[0], refs[0]["spins"][sl])
        c.close()


def test_window_errors():
    m = muca()
    c = m.Context([{"L": 4, "T": 1.0, "n_walkers": 8}], seed=3)
    lo, hi = c.walker_range(0)
    for args in [(hi + 1, hi, 0.0, 0), (-1, hi, 0.0, 0), (lo, 65, 0.0, 0), (lo, hi, 0.5, 0),
                 (lo, hi, -1.0, 1), (lo, hi, float("nan"), 1)]:
        with pytest.raises(m.MucaError) as e:
            c.set_window(0, *args)
        assert e.value.code == m.ERR_INVALID_ARG, args
    with pytest.raises(m.MucaError) as e:  # a walker outside the window
        c.set_window(0, lo + 1, max(hi, lo + 1), 0.0, 0)
    assert e.value.code == m.ERR_WINDOW
    assert c.get_window(0) == (0, 64)
    c.set_window(0, lo, hi, 0.5, 2)
    assert c.get_window(0) == (lo, hi)
    # a state outside the active window is refused and the old state kept
    spins0, _ = c.get_state(0)
    with pytest.raises(m.MucaError) as e:
        c.set_state(0, np.zeros((8, 64), dtype=np.int8))
    assert e.value.code == m.ERR_WINDOW
    assert np.array_equal(c.get_state(0)[0], spins0)
    # the table refuses every move that leaves the window
    t = c.get_table(0)
    assert (t[hi, 2, :] == 0).all() and (t[lo, 0, :] == 0).all()
    assert (t[lo:hi, 2, :] > 0).any()
    c.close()
