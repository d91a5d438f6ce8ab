"""GPU parity of the sweep path against the CPU oracle (bit-exact).

Every comparison is element by element: initial spins, acceptance tables,
per-iteration merged histograms, lnW after each update, final spins and
tallies, recorded time series.  Inputs are seeded; nothing the oracle
consumes comes from the GPU.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1502_07214_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def muca():
    from paper_1502_07214_gb300 import muca as m

    return m


def ctx_of(groups, seed, **kw):
    return muca().Context(groups, seed=seed, **kw)


def gpu_run(groups, seed, n_iter, sweeps, n_meas=0, use_graph=False, lnW=None, **kw):
    c = ctx_of(groups, seed, **kw)
    if lnW is not None:
        for g, l in enumerate(lnW):
            c.set_lnW(g, l)
    hists = [[] for _ in groups]
    lnWs = [[] for _ in groups]
    if use_graph:
        c.run_graph(n_iter, sweeps)
    else:
        for _ in range(n_iter):
            c.sweep_iter(sweeps)
            for g in range(len(groups)):
                hists[g].append(c.get_hist(g))
            c.merge_update()
            for g in range(len(groups)):
                lnWs[g].append(c.get_lnW(g))
    if n_meas:
        c.reserve_timeseries(n_meas)
        c.sweep_iter(n_meas, record=True)
    out = []
    for g in range(len(groups)):
        spins, tal = c.get_state(g)
        out.append({"spins": spins, "tallies": tal, "lnW": c.get_lnW(g),
                    "hist": np.array(hists[g]), "lnWs": lnWs[g],
                    "ts": c.get_timeseries(g) if n_meas else None,
                    "config": c.get_config(g)})
    c.close()
    return out


def walker_offsets(groups):
    off, o = [], 0
    for g in groups:
        off.append(o)
        o += g["n_walkers"]
    return off


def test_initial_spins_and_tallies_match_oracle():
    groups = [{"L": 2, "T": 1.0, "n_walkers": 5}, {"L": 3, "T": 2.0, "n_walkers": 33},
              {"L": 5, "T": 0.9, "n_walkers": 40}, {"L": 8, "T": 1.4182, "n_walkers": 64}]
    c = ctx_of(groups, seed=77)
    for g, (spec, w0) in enumerate(zip(groups, walker_offsets(groups))):
        spins, tal = c.get_state(g)
        for w in range(spec["n_walkers"]):
            ref = oracle.init_spins(spec["L"], 77, w0 + w)
            assert np.array_equal(spins[w], ref), (g, w)
            assert list(tal[w]) == list(oracle.energies(spec["L"], ref))
    c.close()


@pytest.mark.parametrize("L,T", [(2, 1.0), (4, 0.9), (8, 2.0), (16, 1.4182)])
def test_table_bit_exact(L, T):
    V = L ** 3
    c = ctx_of([{"L": L, "T": T, "n_walkers": 32}], seed=1)
    assert np.array_equal(c.get_table(0), oracle.build_table(L, T, 0, V, np.zeros(V + 1)))
    lnW = wl.random_lnW(V + 1, seed=L, scale=2.0, slope=-1.0 / T * 2.8)
    c.set_lnW(0, lnW)
    assert np.array_equal(c.get_table(0), oracle.build_table(L, T, 0, V, lnW))
    c.close()


def test_merge_update_bit_exact_on_a_given_histogram():
    L, T = 6, 1.0
    V = L ** 3
    c = ctx_of([{"L": L, "T": T, "n_walkers": 32}], seed=2)
    lnW0 = wl.random_lnW(V + 1, seed=3)
    c.set_lnW(0, lnW0)
    H = np.random.default_rng(5).integers(0, 1000, V + 1).astype(np.uint64)
    H[::7] = 0
    c.set_hist(0, H)
    c.merge_update()
    ref = lnW0.copy()
    oracle.update_lnW(H, ref)
    assert np.array_equal(c.get_lnW(0), ref)
    assert np.array_equal(c.get_table(0), oracle.build_table(L, T, 0, V, ref))
    assert not c.get_hist(0).any()
    c.close()


def compare_group(got, ref, n_iter):
    assert np.array_equal(got["hist"], ref["hist"][:n_iter])
    assert np.array_equal(got["lnW"], ref["lnW"])
    assert np.array_equal(got["spins"], ref["spins"])
    assert np.array_equal(got["tallies"], ref["tallies"])


@pytest.mark.parametrize("residency,wpb,P", [(1, 32, 1), (1, 16, 2), (1, 8, 4), (1, 4, 8),
                                             (2, 32, 1), (2, 16, 1), (2, 8, 4), (2, 4, 8),
                                             (3, 32, 0), (3, 16, 0), (3, 8, 0), (4, 16, 2),
                                             (0, 0, 0)])
def test_small_workload_full_run_bit_exact(residency, wpb, P):
    """L=8, T=2.0, 64 walkers, 10 iterations x 200 sweeps, seed 0, in full,
    in every kernel configuration (results never depend on it)."""
    s = wl.SMALL
    g = [{"L": s["L"], "T": s["T"], "n_walkers": s["n_walkers"]}]
    got = gpu_run(g, s["seed"], s["n_iter"], s["sweeps"], n_meas=50, residency=residency,
                  walkers_per_block=wpb, lanes_per_walker=P)[0]
    if residency:
        assert got["config"] == (residency, wpb, P)
    ref = oracle.muca_run(s["L"], s["T"], s["n_walkers"], s["seed"], s["n_iter"], s["sweeps"],
                          n_meas=50)
    compare_group(got, ref, s["n_iter"])
    # time series: GPU [sample][field][walker] vs oracle [walker][sample][field]
    assert np.array_equal(got["ts"], ref["ts"].transpose(1, 2, 0))


def test_graph_form_equals_plain_form():
    groups = [{"L": 4, "T": 1.0, "n_walkers": 40}, {"L": 6, "T": 0.9, "n_walkers": 70},
              {"L": 8, "T": 2.0, "n_walkers": 33}]
    a = gpu_run(groups, 9, 4, 25)
    b = gpu_run(groups, 9, 4, 25, use_graph=True)
    for x, y in zip(a, b):
        assert np.array_equal(x["spins"], y["spins"])
        assert np.array_equal(x["tallies"], y["tallies"])
        assert np.array_equal(x["lnW"], y["lnW"])


@pytest.mark.parametrize("residency", [0, 3])
def test_mixed_groups_reduced_bit_exact(residency):
    """The mixed (L, T) batch in one context, few walkers per group (ragged)."""
    groups = wl.mixed_groups(n_walkers=37)
    got = gpu_run(groups, wl.MIXED["seed"], 2, 3, n_meas=2, residency=residency)
    for g, (spec, w0) in enumerate(zip(groups, walker_offsets(groups))):
        ref = oracle.muca_run(spec["L"], spec["T"], spec["n_walkers"], wl.MIXED["seed"], 2, 3,
                              n_meas=2, walker_id0=w0)
        compare_group(got[g], ref, 2)
        assert np.array_equal(got[g]["ts"], ref["ts"].transpose(1, 2, 0))


@pytest.mark.parametrize("P", [1, 2, 8, 0])
def test_generic_and_unrolled_sizes_in_one_launch(P):
    """Sizes of the unrolled row path and of the plain per-site path (L % 4 != 0)
    side by side; lanes per walker apply to the unrolled sizes only."""
    groups = [{"L": L, "T": T, "n_walkers": nw}
              for L, T, nw in [(2, 1.0, 7), (3, 2.0, 33), (4, 0.9, 40), (5, 1.4182, 9),
                               (12, 1.0, 65), (20, 2.0, 31)]]
    got = gpu_run(groups, 23, 2, 4, n_meas=3, residency=1 if P else 3, lanes_per_walker=P)
    for g, (spec, w0) in enumerate(zip(groups, walker_offsets(groups))):
        ref = oracle.muca_run(spec["L"], spec["T"], spec["n_walkers"], 23, 2, 4, n_meas=3,
                              walker_id0=w0)
        compare_group(got[g], ref, 2)
        assert np.array_equal(got[g]["ts"], ref["ts"].transpose(1, 2, 0))


@pytest.mark.parametrize("use_graph", [False, True])
def test_narrow_and_wide_split_kernels_in_one_context(use_graph):
    """Split residency over rows of 8..32 sites (register-carry helpers) and of
    48 sites (rolled helpers), plus a size the split kernel does not cover
    (L = 5, lanes-per-walker kernel): three launches of one iteration, ragged
    walker counts, plain and graph form."""
    groups = [{"L": L, "T": T, "n_walkers": nw}
              for L, T, nw in [(48, 0.9, 19), (8, 2.0, 40), (5, 1.0, 7), (32, 1.4182, 9),
                               (12, 1.0, 33)]]
    seed, n_iter, sweeps = 29, 2, 2
    got = gpu_run(groups, seed, n_iter, sweeps, n_meas=2, use_graph=use_graph, residency=3)
    for g, (spec, w0) in enumerate(zip(groups, walker_offsets(groups))):
        assert got[g]["config"][0] == (3 if spec["L"] % 4 == 0 else 1), spec
        ref = oracle.muca_run(spec["L"], spec["T"], spec["n_walkers"], seed, n_iter, sweeps,
                              n_meas=2, walker_id0=w0)
        if use_graph:
            assert np.array_equal(got[g]["lnW"], ref["lnW"])
            assert np.array_equal(got[g]["spins"], ref["spins"])
            assert np.array_equal(got[g]["tallies"], ref["tallies"])
        else:
            compare_group(got[g], ref, n_iter)
        assert np.array_equal(got[g]["ts"], ref["ts"].transpose(1, 2, 0))


def test_largest_sizes_per_site_path():
    """Row lengths the unrolled paths do not take (44, and 52 up to the
    maximum L = 64, V = 262144 sites) run on the per-site path with the
    global table: spins, tallies, weights and series bit-exact."""
    groups = [{"L": L, "T": T, "n_walkers": nw}
              for L, T, nw in [(44, 1.0, 3), (52, 0.9, 2), (64, 0.9, 5)]]
    assert max(g["L"] for g in groups) == muca().MAX_L
    got = gpu_run(groups, 17, 2, 1, n_meas=1)
    for g, (spec, w0) in enumerate(zip(groups, walker_offsets(groups))):
        ref = oracle.muca_run(spec["L"], spec["T"], spec["n_walkers"], 17, 2, 1, n_meas=1,
                              walker_id0=w0)
        compare_group(got[g], ref, 2)
        assert np.array_equal(got[g]["ts"], ref["ts"].transpose(1, 2, 0))


def test_medium_workload_reduced_bit_exact():
    """L=16, T=1.0, 1024 walkers, seed 1: 2 iterations x 8 sweeps + 4 measured."""
    s = wl.MEDIUM
    g = [{"L": s["L"], "T": s["T"], "n_walkers": s["n_walkers"]}]
    got = gpu_run(g, s["seed"], 2, 8, n_meas=4)[0]
    ref = oracle.muca_run(s["L"], s["T"], s["n_walkers"], s["seed"], 2, 8, n_meas=4)
    compare_group(got, ref, 2)
    assert np.array_equal(got["ts"], ref["ts"].transpose(1, 2, 0))


def sample_walkers(W):
    return sorted({0, 1, 31, 32, 33, W // 2, W - 33, W - 1} & set(range(W)))


@pytest.mark.parametrize("residency,P", [(0, 0), (1, 4), (1, 8), (3, 0), (4, 0)])
def test_large_workload_full_size_sampled_walkers(residency, P):
    """L=48, T=0.9, all 4096 walkers in the benchmark's launch configuration,
    under a fixed non-trivial weight: sampled walkers recomputed by the oracle,
    plus the merged histogram against the recorded series (any size)."""
    s = wl.LARGE
    L, T, W = s["L"], s["T"], s["n_walkers"]
    V = L ** 3
    lnW = wl.random_lnW(V + 1, seed=11, scale=0.3, slope=-2.9 / T)
    c = ctx_of([{"L": L, "T": T, "n_walkers": W}], seed=s["seed"], residency=residency,
               lanes_per_walker=P)
    c.set_lnW(0, lnW)
    n = 2
    c.reserve_timeseries(n)
    c.sweep_iter(n, record=True)
    spins, tal = c.get_state(0)
    ts = c.get_timeseries(0)
    H = c.get_hist(0)
    c.close()
    thr = oracle.build_table(L, T, 0, V, lnW)
    for w in sample_walkers(W):
        sp = oracle.init_spins(L, s["seed"], w)
        t = oracle.energies(L, sp).astype(np.int32)
        ref_ts = oracle.sweeps(L, 0, V, thr, s["seed"], w, 0, n, sp, t, record=True)
        assert np.array_equal(spins[w], sp), w
        assert np.array_equal(tal[w], t), w
        assert np.array_equal(ts[:, :, w], ref_ts), w
    # property at any size: the histogram is the count of recorded E_Delta values
    want = np.bincount(ts[:, 1, :].ravel(), minlength=V + 1).astype(np.uint64)
    assert np.array_equal(H, want)
    assert H.sum() == n * W


def test_mixed_workload_full_size_sampled_walkers():
    """All 24 (L, T) groups x 512 walkers in one graph iteration: sampled
    walkers of every group against the oracle; histogram totals."""
    groups = wl.mixed_groups()
    seed = wl.MIXED["seed"]
    c = ctx_of(groups, seed)
    n = 2
    c.reserve_timeseries(n)
    c.sweep_iter(n, record=True)
    offs = walker_offsets(groups)
    for g, spec in enumerate(groups):
        L, T, W = spec["L"], spec["T"], spec["n_walkers"]
        V = L ** 3
        spins, tal = c.get_state(g)
        ts = c.get_timeseries(g)
        assert c.get_hist(g).sum() == n * W
        thr = oracle.build_table(L, T, 0, V, np.zeros(V + 1))
        for w in (0, 255, 511):
            sp = oracle.init_spins(L, seed, offs[g] + w)
            t = oracle.energies(L, sp).astype(np.int32)
            ref_ts = oracle.sweeps(L, 0, V, thr, seed, offs[g] + w, 0, n, sp, t, record=True)
            assert np.array_equal(spins[w], sp) and np.array_equal(ts[:, :, w], ref_ts), (g, w)
    c.close()


def test_restricted_window_and_set_state():
    L, T, W = 5, 1.0, 40
    V = L ** 3
    e_min, e_max = 40, 90
    rng = np.random.default_rng(8)
    spins = np.zeros((W, V), dtype=np.int8)
    for w in range(W):
        idx = rng.choice(V, 60, replace=False)
        spins[w, idx] = rng.choice(np.array([-1, 1], dtype=np.int8), 60)
    groups = [{"L": L, "T": T, "n_walkers": W, "e_min": e_min, "e_max": e_max}]
    c = ctx_of(groups, seed=4)
    c.set_state(0, spins)
    lnW = wl.random_lnW(e_max - e_min + 1, seed=2)
    c.set_lnW(0, lnW)
    c.reserve_timeseries(30)
    c.sweep_iter(30, record=True)
    g_spins, g_tal = c.get_state(0)
    ts = c.get_timeseries(0)
    sweep0 = 0
    thr = oracle.build_table(L, T, e_min, e_max, lnW)
    for w in range(W):
        sp = spins[w].copy()
        t = oracle.energies(L, sp).astype(np.int32)
        ref = oracle.sweeps(L, e_min, e_max, thr, 4, w, sweep0, 30, sp, t, record=True)
        assert np.array_equal(g_spins[w], sp) and np.array_equal(ts[:, :, w], ref)
    assert ts[:, 1, :].min() >= e_min and ts[:, 1, :].max() <= e_max
    bad = spins.copy()
    bad[0, :] = 0  # E_Delta = 0 < e_min
    with pytest.raises(muca().MucaError) as e:
        c.set_state(0, bad)
    assert e.value.code == muca().ERR_WINDOW
    bad = spins.copy()
    bad[0, 0] = 2
    with pytest.raises(muca().MucaError) as e:
        c.set_state(0, bad)
    assert e.value.code == muca().ERR_INVALID_ARG
    # the rejected states left the context unchanged
    s2, t2 = c.get_state(0)
    assert np.array_equal(s2, g_spins) and np.array_equal(t2, g_tal)
    c.close()


@pytest.mark.parametrize("e_min,e_max,res,P", [(300, 320, 1, 1), (250, 350, 1, 4),
                                              (420, 512, 1, 8), (250, 350, 3, 0),
                                              (420, 512, 3, 0), (250, 350, 4, 0),
                                              (420, 512, 4, 0), (300, 312, 4, 0)])
def test_restricted_window_unrolled_size(e_min, e_max, res, P):
    """L=8 with a restricted E_Delta window: a window narrower than the kernel's
    table window (plain path) and wider ones that reach the top of the range
    (unrolled path, table window clamped to the window's rows)."""
    L, T, W = 8, 1.0, 24
    V = L ** 3
    rng = np.random.default_rng(e_min)
    spins = np.zeros((W, V), dtype=np.int8)
    for w in range(W):
        n = int(rng.integers(e_min, e_max + 1))
        idx = rng.choice(V, n, replace=False)
        spins[w, idx] = rng.choice(np.array([-1, 1], dtype=np.int8), n)
    c = ctx_of([{"L": L, "T": T, "n_walkers": W, "e_min": e_min, "e_max": e_max}], seed=31,
               residency=res, lanes_per_walker=P)
    c.set_state(0, spins)
    lnW = wl.random_lnW(e_max - e_min + 1, seed=e_max, scale=0.8)
    c.set_lnW(0, lnW)
    c.reserve_timeseries(25)
    c.sweep_iter(25, record=True)
    g_spins, _ = c.get_state(0)
    ts = c.get_timeseries(0)
    c.close()
    thr = oracle.build_table(L, T, e_min, e_max, lnW)
    for w in range(W):
        sp = spins[w].copy()
        t = oracle.energies(L, sp).astype(np.int32)
        ref = oracle.sweeps(L, e_min, e_max, thr, 31, w, 0, 25, sp, t, record=True)
        assert np.array_equal(g_spins[w], sp) and np.array_equal(ts[:, :, w], ref), w


def test_ising_limit_on_gpu():
    """Delta -> -inf: from all-(+-1) states no vacancy is ever created."""
    L, T, W = 4, 1.8, 64
    V = L ** 3
    c = ctx_of([{"L": L, "T": T, "n_walkers": W}], seed=6)
    rng = np.random.default_rng(6)
    c.set_state(0, rng.choice(np.array([-1, 1], dtype=np.int8), size=(W, V)))
    c.set_lnW(0, -(1.0 / T) * (-1e6) * np.arange(V + 1))
    c.reserve_timeseries(50)
    c.sweep_iter(50, record=True)
    ts = c.get_timeseries(0)
    assert (ts[:, 1, :] == V).all()
    c.close()


def test_tally_check_and_checkpoint_restore(tmp_path):
    groups = [{"L": 6, "T": 1.0, "n_walkers": 50}, {"L": 3, "T": 2.0, "n_walkers": 9}]
    c = ctx_of(groups, seed=12, debug_flags=1)
    c.sweep_iter(5)
    c.merge_update()
    c.sweep_iter(3)
    c.check_tallies()
    path = str(tmp_path / "ck.bin")
    c.checkpoint(path)
    c.sweep_iter(7)
    c.merge_update()
    c.sweep_iter(4)
    a = [c.get_state(g) for g in range(2)]
    la = [c.get_lnW(g) for g in range(2)]
    c.close()
    d = ctx_of(groups, seed=12)
    d.restore(path)
    assert d.sweep_count() == 8
    d.sweep_iter(7)
    d.merge_update()
    d.sweep_iter(4)
    for g in range(2):
        s, t = d.get_state(g)
        assert np.array_equal(s, a[g][0]) and np.array_equal(t, a[g][1])
        assert np.array_equal(d.get_lnW(g), la[g])
    d.close()


def test_errors_are_reported_not_raised_as_faults():
    c = ctx_of([{"L": 4, "T": 1.0, "n_walkers": 32}], seed=1)
    with pytest.raises(muca().MucaError) as e:
        c.sweep_iter(3, record=True)  # no time series reserved
    assert e.value.code == muca().ERR_INVALID_ARG
    with pytest.raises(muca().MucaError) as e:
        c.get_lnW(5)
    assert e.value.code == muca().ERR_INVALID_ARG
    with pytest.raises(muca().MucaError) as e:
        c.set_table(3, oracle.build_table(4, 1.0, 0, 64, np.zeros(65)))
    assert e.value.code == muca().ERR_INVALID_ARG
    with pytest.raises(muca().MucaError) as e:
        c.run_graph(-1, 5)
    assert e.value.code == muca().ERR_INVALID_ARG
    # d = 0 moves do not change E_Delta, so their thresholds cannot depend on it
    t = oracle.build_table(4, 1.0, 0, 64, np.zeros(65))
    t[3, 1, 0] ^= 1
    with pytest.raises(muca().MucaError) as e:
        c.set_table(0, t)
    assert e.value.code == muca().ERR_INVALID_ARG
    c.close()


def test_injected_table_is_used():
    """A table given through muca_set_table drives the sweeps (the oracle gets
    the same table)."""
    L, T, W = 4, 1.3, 32
    V = L ** 3
    lnW = wl.random_lnW(V + 1, seed=21, scale=1.5)
    thr = oracle.build_table(L, T, 0, V, lnW)
    c = ctx_of([{"L": L, "T": T, "n_walkers": W}], seed=5)
    c.set_table(0, thr)
    assert np.array_equal(c.get_table(0), thr)
    c.sweep_iter(20)
    spins, tal = c.get_state(0)
    for w in range(W):
        sp = oracle.init_spins(L, 5, w)
        t = oracle.energies(L, sp).astype(np.int32)
        oracle.sweeps(L, 0, V, thr, 5, w, 0, 20, sp, t)
        assert np.array_equal(spins[w], sp)
    c.close()


@pytest.mark.parametrize("use_graph", [False, True])
def test_row_scan_kernel_every_shape_in_one_context(use_graph):
    """The row-scan kernel over its range of row lengths (segments of 1, 2, 4,
    8 and 16 lanes per walker, with idle lanes where L / 4 is not a power of
    2), ragged walker counts (partial warps and blocks) and several warps per
    block, plus a size it does not cover (L = 10, falls back to the
    lanes-per-walker kernel): weights after two iterations, recorded series,
    plain and graph form, against the oracle."""
    groups = [{"L": L, "T": T, "n_walkers": nw}
              for L, T, nw in [(4, 1.0, 35), (8, 2.0, 37), (12, 1.4182, 23), (16, 1.0, 9),
                               (20, 0.9, 14), (24, 1.0, 21), (28, 2.0, 5), (32, 0.9, 11),
                               (36, 1.0, 3), (48, 0.9, 9), (64, 0.9, 3), (10, 1.0, 7)]]
    seed, n_iter, sweeps = 41, 2, 3
    got = gpu_run(groups, seed, n_iter, sweeps, n_meas=3, use_graph=use_graph, residency=4)
    for g, (spec, w0) in enumerate(zip(groups, walker_offsets(groups))):
        want_res = 4 if spec["L"] != 10 else 1
        assert got[g]["config"][0] == want_res, spec
        ref = oracle.muca_run(spec["L"], spec["T"], spec["n_walkers"], seed, n_iter, sweeps,
                              n_meas=3, walker_id0=w0)
        if use_graph:
            assert np.array_equal(got[g]["lnW"], ref["lnW"])
            assert np.array_equal(got[g]["spins"], ref["spins"])
            assert np.array_equal(got[g]["tallies"], ref["tallies"])
        else:
            compare_group(got[g], ref, n_iter)
        assert np.array_equal(got[g]["ts"], ref["ts"].transpose(1, 2, 0)), spec


@pytest.mark.parametrize("L,T,delta", [(8, 0.9, 2.964), (16, 0.9, 2.964), (24, 1.0, 2.944),
                                       (48, 0.9, 2.964)])
def test_row_scan_kernel_under_transition_weights(L, T, delta):
    """Canonical weights at the first-order transition field from a random
    start: many accepted moves that change E_Delta per row, so rows are
    resolved in several segments and the table window moves often."""
    V = L ** 3
    W = 40
    lnW = -(1.0 / T) * delta * np.arange(V + 1)
    c = ctx_of([{"L": L, "T": T, "n_walkers": W}], seed=L, residency=4)
    c.set_lnW(0, lnW)
    n = 12
    c.reserve_timeseries(n)
    c.sweep_iter(n, record=True)
    spins, tal = c.get_state(0)
    ts = c.get_timeseries(0)
    assert c.get_config(0)[0] == 4
    c.close()
    thr = oracle.build_table(L, T, 0, V, lnW)
    for w in range(W):
        sp = oracle.init_spins(L, L, w)
        t = oracle.energies(L, sp).astype(np.int32)
        ref = oracle.sweeps(L, 0, V, thr, L, w, 0, n, sp, t, record=True)
        assert np.array_equal(spins[w], sp) and np.array_equal(tal[w], t), w
        assert np.array_equal(ts[:, :, w], ref), w
