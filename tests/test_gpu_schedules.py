"""GPU parity on the workloads' own schedules (bit-exact against the oracle).

The other GPU tests check the sweep on short runs; these follow the
configurations' full iteration schedules, where the walkers reach the
converged, flat-histogram regime and the E_Delta window of each walker moves
the most:
  - the medium workload (L=16, T=1.0, 1024 walkers, 30 x 500 sweeps, seed 1)
    in full, every walker, against one whole oracle run;
  - the large workload (L=48, T=0.9, 4096 walkers, seed 3) in the benchmark's
    launch configuration: a short schedule with every walker against one whole
    oracle run, and three full 1000-sweep iterations plus 250 recorded sweeps
    with sampled walkers replayed by the oracle under the weights of each
    iteration;
  - the large workload under canonical weights at the transition field
    (Delta = 2.964, T = 0.9), the vacancy-rich regime in which a walker's
    E_Delta moves by several bins within a row;
  - the mixed workload (24 groups x 512 walkers, seed 2), five 300-sweep
    iterations, in plain and graph form.

Where the oracle replays only sampled walkers, the weights of each iteration
follow from the merged histogram of all 4096 walkers, which only the device
run has.  The oracle then takes that histogram as data: it applies its own
weight recursion to it (compared with the device's lnW), builds its own
tables from the result and replays the sampled walkers from their initial
spins.  The histogram is checked by what holds at any size (its total, and
equality with the count of the recorded E_Delta values).  The all-walker runs
need no such input.
"""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
from paper_1502_07214_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

THREADS = os.cpu_count() or 1


def muca():
    from paper_1502_07214_gb300 import muca as m

    return m


def spread_walkers(W, block=16, n=24):
    """Walkers spread over blocks and warps: the first and last of the first
    blocks, block boundaries, and evenly spaced ones."""
    pick = {0, 1, block - 1, block, block + 1, 31, 32, W // 2 - 1, W // 2, W - 2, W - 1}
    pick |= set(np.linspace(0, W - 1, n - len(pick) + 2).astype(int).tolist())
    return sorted(w for w in pick if 0 <= w < W)


def replay(L, T, seed, walkers, stages, e_min=0, e_max=None):
    """Oracle replay of sampled walkers from their initial spins through
    stages of (lnW, n_sweeps, record); each stage's table is built by the
    oracle from lnW.  Walkers run in threads (the oracle releases the GIL).
    Returns {walker: (spins, tallies, series of the recorded stages)}."""
    V = L ** 3
    e_max = V if e_max is None else e_max
    tables = [oracle.build_table(L, T, e_min, e_max, lnW) for lnW, _, _ in stages]

    def one(w):
        sp = oracle.init_spins(L, seed, w)
        t = oracle.energies(L, sp).astype(np.int32)
        sweep0, series = 0, []
        for thr, (_, n, rec) in zip(tables, stages):
            ts = oracle.sweeps(L, e_min, e_max, thr, seed, w, sweep0, n, sp, t, record=rec)
            if rec:
                series.append(ts)
            sweep0 += n
        return w, (sp, t, np.concatenate(series) if series else None)

    with ThreadPoolExecutor(THREADS) as ex:
        return dict(ex.map(one, walkers))


def test_medium_workload_full_schedule_every_walker():
    """L=16, T=1.0, 1024 walkers, 30 iterations x 500 sweeps, seed 1, then 100
    recorded sweeps: every merged histogram, the final lnW, the spins, the
    tallies and the series of every walker equal one oracle run."""
    s = wl.MEDIUM
    n_meas = 100
    c = muca().Context([{"L": s["L"], "T": s["T"], "n_walkers": s["n_walkers"]}], seed=s["seed"])
    hists = []
    for _ in range(s["n_iter"]):
        c.sweep_iter(s["sweeps"])
        hists.append(c.get_hist(0))
        c.merge_update()
    c.reserve_timeseries(n_meas)
    c.sweep_iter(n_meas, record=True)
    spins, tal = c.get_state(0)
    lnW, ts = c.get_lnW(0), c.get_timeseries(0)
    c.close()
    ref = oracle.muca_run(s["L"], s["T"], s["n_walkers"], s["seed"], s["n_iter"], s["sweeps"],
                          n_meas=n_meas)
    for it in range(s["n_iter"]):
        assert np.array_equal(hists[it], ref["hist"][it]), f"histogram of iteration {it}"
    assert np.array_equal(lnW, ref["lnW"])
    assert np.array_equal(spins, ref["spins"])
    assert np.array_equal(tal, ref["tallies"])
    assert np.array_equal(ts, ref["ts"].transpose(1, 2, 0))
    # the run left the random start: the last histogram covers a wide range
    assert (ref["hist"][-1] > 0).sum() > 200


def test_large_workload_short_schedule_every_walker():
    """L=48, T=0.9, all 4096 walkers in the benchmark's launch configuration:
    3 iterations x 12 sweeps then 8 recorded sweeps, every walker and every
    merged histogram against one whole oracle run."""
    s = wl.LARGE
    L, T, W = s["L"], s["T"], s["n_walkers"]
    n_iter, sweeps, n_meas = 3, 12, 8
    c = muca().Context([{"L": L, "T": T, "n_walkers": W}], seed=s["seed"])
    hists = []
    for _ in range(n_iter):
        c.sweep_iter(sweeps)
        hists.append(c.get_hist(0))
        c.merge_update()
    c.reserve_timeseries(n_meas)
    c.sweep_iter(n_meas, record=True)
    spins, tal = c.get_state(0)
    lnW, ts = c.get_lnW(0), c.get_timeseries(0)
    c.close()
    ref = oracle.muca_run(L, T, W, s["seed"], n_iter, sweeps, n_meas=n_meas)
    for it in range(n_iter):
        assert np.array_equal(hists[it], ref["hist"][it]), f"histogram of iteration {it}"
    assert np.array_equal(lnW, ref["lnW"])
    assert np.array_equal(tal, ref["tallies"])
    assert np.array_equal(spins, ref["spins"])
    assert np.array_equal(ts, ref["ts"].transpose(1, 2, 0))


def test_large_workload_full_iterations_sampled_walkers():
    """L=48, T=0.9, 4096 walkers, seed 3: three full iterations of 1000 sweeps
    (merge, FP64 update and table rebuild after each), then 250 recorded
    sweeps, in the benchmark's launch configuration.  24 sampled walkers are
    replayed by the oracle through the same schedule; the device's weight
    update equals the oracle's on each merged histogram."""
    s = wl.LARGE
    L, T, W = s["L"], s["T"], s["n_walkers"]
    V = L ** 3
    n_iter, sweeps, n_meas = 3, s["sweeps"], s["n_meas"] // s["n_iter"]
    c = muca().Context([{"L": L, "T": T, "n_walkers": W}], seed=s["seed"])
    res, wpb, _ = c.get_config(0)
    lnWs = [np.zeros(V + 1)]
    for it in range(n_iter):
        c.sweep_iter(sweeps)
        H = c.get_hist(0)
        assert H.sum() == W * sweeps
        c.merge_update()
        got = c.get_lnW(0)
        want = lnWs[-1].copy()
        oracle.update_lnW(H, want)
        assert np.array_equal(got, want), f"weight update of iteration {it}"
        assert np.array_equal(c.get_table(0), oracle.build_table(L, T, 0, V, want))
        lnWs.append(got)
    c.reserve_timeseries(n_meas)
    c.sweep_iter(n_meas, record=True)
    spins, tal = c.get_state(0)
    ts = c.get_timeseries(0)
    H = c.get_hist(0)
    c.close()
    want_h = np.bincount(ts[:, 1, :].ravel(), minlength=V + 1).astype(np.uint64)
    assert np.array_equal(H, want_h)
    stages = [(lnWs[i], sweeps, False) for i in range(n_iter)] + [(lnWs[-1], n_meas, True)]
    walkers = spread_walkers(W, block=max(wpb, 1))
    assert len(walkers) >= 16
    ref = replay(L, T, s["seed"], walkers, stages)
    for w in walkers:
        sp, t, rts = ref[w]
        assert np.array_equal(spins[w], sp), w
        assert np.array_equal(tal[w], t), w
        assert np.array_equal(ts[:, :, w], rts), w


def test_large_workload_vacancy_rich_transition_weights():
    """L=48, T=0.9, 4096 walkers under canonical weights at the first-order
    transition field (lnW = -beta Delta E_Delta, Delta = 2.964): from the
    random start the walkers' E_Delta moves by several bins within a row, so
    the table window is re-centred often and rows whose E_Delta left it are
    redone from the global table.  60 recorded sweeps; sampled walkers against
    the oracle, the histogram against the series."""
    s = wl.LARGE
    L, T, W = s["L"], s["T"], s["n_walkers"]
    V = L ** 3
    n = 60
    lnW = -(1.0 / T) * 2.964 * np.arange(V + 1)
    c = muca().Context([{"L": L, "T": T, "n_walkers": W}], seed=s["seed"] + 100)
    _, wpb, _ = c.get_config(0)
    c.set_lnW(0, lnW)
    c.reserve_timeseries(n)
    c.sweep_iter(n, record=True)
    spins, tal = c.get_state(0)
    ts = c.get_timeseries(0)
    H = c.get_hist(0)
    c.close()
    assert np.array_equal(H, np.bincount(ts[:, 1, :].ravel(), minlength=V + 1).astype(np.uint64))
    # the regime: the walkers fall into the vacancy-rich phase (E_Delta near
    # V / 10) and E_Delta still moves by about a hundred bins per sweep there
    steps = np.abs(np.diff(ts[:, 1, :].astype(np.int64), axis=0))
    assert np.median(ts[-1, 1, :]) < V // 4
    assert np.median(steps) > 30
    walkers = spread_walkers(W, block=max(wpb, 1))
    ref = replay(L, T, s["seed"] + 100, walkers, [(lnW, n, True)])
    for w in walkers:
        sp, t, rts = ref[w]
        assert np.array_equal(spins[w], sp), w
        assert np.array_equal(tal[w], t), w
        assert np.array_equal(ts[:, :, w], rts), w


def test_mixed_workload_five_iterations_plain_and_graph():
    """24 groups (L in {8,...,32} x T in {2.0, 1.4182, 1.0, 0.9}) x 512
    walkers, seed 2, five iterations x 300 sweeps: the graph form equals the
    plain form for every walker; in the plain form, every weight update equals
    the oracle's on the merged histogram, and three walkers per group (first,
    middle, last) are replayed by the oracle through the five iterations."""
    groups = wl.mixed_groups()
    seed, n_iter, sweeps = wl.MIXED["seed"], 5, wl.MIXED["sweeps"]
    offs = np.cumsum([0] + [g["n_walkers"] for g in groups])[:-1]
    plain = muca().Context(groups, seed=seed)
    lnWs = [[np.zeros(g["L"] ** 3 + 1)] for g in groups]
    for it in range(n_iter):
        plain.sweep_iter(sweeps)
        Hs = [plain.get_hist(g) for g in range(len(groups))]
        plain.merge_update()
        for g, spec in enumerate(groups):
            assert Hs[g].sum() == spec["n_walkers"] * sweeps
            want = lnWs[g][-1].copy()
            oracle.update_lnW(Hs[g], want)
            got = plain.get_lnW(g)
            assert np.array_equal(got, want), (g, it)
            lnWs[g].append(got)
    p_state = [plain.get_state(g) for g in range(len(groups))]
    plain.close()
    graph = muca().Context(groups, seed=seed)
    graph.run_graph(n_iter, sweeps)
    for g in range(len(groups)):
        s, t = graph.get_state(g)
        assert np.array_equal(s, p_state[g][0]), g
        assert np.array_equal(t, p_state[g][1]), g
        assert np.array_equal(graph.get_lnW(g), lnWs[g][-1]), g
    graph.close()
    for g, spec in enumerate(groups):
        L, T = spec["L"], spec["T"]
        stages = [(lnWs[g][i], sweeps, False) for i in range(n_iter)]
        ids = [int(offs[g]) + w for w in (0, 255, 511)]
        ref = replay(L, T, seed, ids, stages)
        for w in (0, 255, 511):
            sp, t, _ = ref[int(offs[g]) + w]
            assert np.array_equal(p_state[g][0][w], sp), (g, w)
            assert np.array_equal(p_state[g][1][w], t), (g, w)
