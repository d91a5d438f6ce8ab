"""The disordered model (the oracle's reading R16: one quenched integer
coupling per bond) on the GPU, against the oracle, bit for bit: per-iteration
histograms, weights, spins, tallies and recorded series of groups with
bimodal, +-J and diluted couplings beside a clean group in one context, in
the plain and the graph form, with the accumulated recursion and an adaptive
window, through a checkpoint, and in the row-scan-free one-thread-per-walker
kernel that such groups run.
"""
import numpy as np
import pytest

import oracle
from paper_1502_07214_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

SEED, N_ITER, SWEEPS, N_MEAS = 17, 4, 40, 9
# (group, couplings (j1, j2) or None for the clean model)
GROUPS = [({"L": 4, "T": 3.0, "n_walkers": 40}, (1, 3)),
          ({"L": 6, "T": 1.5, "n_walkers": 33}, (-1, 1)),
          ({"L": 8, "T": 2.0, "n_walkers": 37}, (0, 2)),
          ({"L": 8, "T": 2.0, "n_walkers": 20}, None),
          ({"L": 5, "T": 4.0, "n_walkers": 9}, (2, 5))]


def muca():
    from paper_1502_07214_gb300 import muca as m

    return m


def bonds_of(i, spec, jj):
    return None if jj is None else wl.random_bonds(spec["L"], jj[0], jj[1], seed=100 + i)


def oracle_runs(groups, recursion=0, n_iter=N_ITER, windows=None, grow=(0.0, 0)):
    out, id0 = [], 0
    for i, (spec, jj) in enumerate(groups):
        kw = {}
        if windows is not None:
            kw = dict(window=windows[i], grow_flat=grow[0], grow_step=grow[1])
        out.append(oracle.muca_run(spec["L"], spec["T"], spec["n_walkers"], SEED, n_iter, SWEEPS,
                                   n_meas=N_MEAS, walker_id0=id0, bonds=bonds_of(i, spec, jj),
                                   recursion=recursion, **kw))
        id0 += spec["n_walkers"]
    return out


def context(groups, recursion=0, **kw):
    c = muca().Context([g for g, _ in groups], seed=SEED, **kw)
    c.set_recursion(recursion)
    for i, (spec, jj) in enumerate(groups):
        J = bonds_of(i, spec, jj)
        if J is not None:
            c.set_bonds(i, J)
            assert c.get_config(i)[0] == muca().RES_BONDS
    return c


def check(c, refs):
    for i, ref in enumerate(refs):
        spins, tal = c.get_state(i)
        assert np.array_equal(c.get_lnW(i), ref["lnW"]), i
        assert np.array_equal(spins, ref["spins"]), i
        assert np.array_equal(tal, ref["tallies"]), i
        assert np.array_equal(c.get_timeseries(i), ref["ts"].transpose(1, 2, 0)), i


def test_initial_tallies_follow_the_couplings():
    c = context(GROUPS)
    for i, (spec, jj) in enumerate(GROUPS):
        spins, tal = c.get_state(i)
        J = bonds_of(i, spec, jj)
        for w in range(0, spec["n_walkers"], 5):
            e = (oracle.energies(spec["L"], spins[w]) if J is None
                 else oracle.energies_bonds(spec["L"], spins[w], J))
            assert tuple(e) == tuple(tal[w]), (i, w)
    c.check_tallies()
    c.close()


@pytest.mark.parametrize("recursion", [0, 1])
def test_plain_form_every_iteration(recursion):
    refs = oracle_runs(GROUPS, recursion)
    c = context(GROUPS, recursion)
    for it in range(N_ITER):
        c.sweep_iter(SWEEPS)
        for i in range(len(GROUPS)):
            assert np.array_equal(c.get_hist(i), refs[i]["hist"][it]), (it, i)
        c.merge_update()
    c.reserve_timeseries(N_MEAS)
    c.sweep_iter(N_MEAS, record=True)
    check(c, refs)
    c.close()


def test_graph_form_and_tally_check():
    refs = oracle_runs(GROUPS)
    c = context(GROUPS, debug_flags=muca().DEBUG_TALLY_CHECK)
    c.run_graph(N_ITER, SWEEPS)
    c.reserve_timeseries(N_MEAS)
    c.sweep_iter(N_MEAS, record=True)
    check(c, refs)
    c.close()


def test_unit_couplings_equal_the_clean_kernels():
    """J = 1 through the disordered kernel equals the clean group in its own
    (autotuned) kernel and the clean oracle."""
    spec = {"L": 8, "T": 1.4182, "n_walkers": 45}
    ref = oracle.muca_run(8, 1.4182, 45, SEED, N_ITER, SWEEPS, n_meas=N_MEAS)
    a = muca().Context([spec], seed=SEED)
    b = muca().Context([spec], seed=SEED)
    b.set_bonds(0, np.ones((512, 3), dtype=np.int8))
    for c in (a, b):
        c.run_graph(N_ITER, SWEEPS)
        c.reserve_timeseries(N_MEAS)
        c.sweep_iter(N_MEAS, record=True)
        check(c, [ref])
        c.close()


def test_adaptive_window_with_couplings():
    groups = GROUPS[:3]
    wins = []
    id0 = 0
    for i, (spec, jj) in enumerate(groups):
        J = bonds_of(i, spec, jj)
        e = [int(oracle.energies_bonds(spec["L"], oracle.init_spins(spec["L"], SEED, id0 + w), J)[1])
             for w in range(spec["n_walkers"])]
        wins.append((min(e), max(e)))
        id0 += spec["n_walkers"]
    refs = oracle_runs(groups, 1, n_iter=12, windows=wins, grow=(0.3, 3))
    c = context(groups, 1)
    for i in range(len(groups)):
        assert c.walker_range(i) == wins[i]
        c.set_window(i, wins[i][0], wins[i][1], 0.3, 3)
    c.run_graph(12, SWEEPS)
    c.reserve_timeseries(N_MEAS)
    c.sweep_iter(N_MEAS, record=True)
    check(c, refs)
    for i in range(len(groups)):
        assert c.get_window(i) == tuple(int(x) for x in refs[i]["windows"][-1])
    c.close()


def test_checkpoint_carries_the_couplings(tmp_path):
    path = str(tmp_path / "bonds.ck")
    a = context(GROUPS)
    a.sweep_iter(SWEEPS)
    a.merge_update()
    a.checkpoint(path)
    a.sweep_iter(SWEEPS)
    a.merge_update()
    b = muca().Context([g for g, _ in GROUPS], seed=SEED)  # clean until the restore
    b.restore(path)
    for i, (_, jj) in enumerate(GROUPS):
        assert (b.get_config(i)[0] == muca().RES_BONDS) == (jj is not None), i
    b.sweep_iter(SWEEPS)
    b.merge_update()
    for i in range(len(GROUPS)):
        assert np.array_equal(b.get_lnW(i), a.get_lnW(i)), i
        assert np.array_equal(b.get_state(i)[0], a.get_state(i)[0]), i
        assert np.array_equal(b.get_state(i)[1], a.get_state(i)[1]), i
    a.close()
    b.close()


def test_bond_errors_and_return_to_the_clean_model():
    m = muca()
    c = m.Context([{"L": 4, "T": 2.0, "n_walkers": 8}], seed=3)
    J = wl.random_bonds(4, 1, 3, seed=1)
    for args in [(J, 2), (J, 0), (J, 9)]:
        with pytest.raises(m.MucaError) as e:
            c.set_bonds(0, *args)
        assert e.value.code == m.ERR_INVALID_ARG
    c.set_bonds(0, J)
    with pytest.raises(m.MucaError) as e:
        c.get_table(0)
    assert e.value.code == m.ERR_INVALID_ARG
    spins, tal = c.get_state(0)
    assert tuple(tal[0]) == tuple(oracle.energies_bonds(4, spins[0], J))
    c.set_bonds(0, None)
    spins, tal = c.get_state(0)
    assert tuple(tal[0]) == tuple(oracle.energies(4, spins[0]))
    assert c.get_config(0)[0] != m.RES_BONDS
    c.get_table(0)
    c.close()


def test_disordered_workload_full_size_sampled_walkers():
    """The benchmark's disordered workload (4096 walkers of L = 24, bimodal
    couplings 5 / 3) in its launch configuration: three recorded sweeps of
    every walker on the GPU; sampled walkers (first, last, ragged middle)
    against the oracle run of the same global walker ids, and the histogram
    against the recorded series."""
    d = wl.DISORDERED
    L, W = d["L"], d["n_walkers"]
    J = wl.random_bonds(L, d["j1"], d["j2"], seed=d["bond_seed"])
    c = muca().Context([{"L": L, "T": d["T"], "n_walkers": W}], seed=d["seed"])
    c.set_bonds(0, J)
    c.reserve_timeseries(3)
    c.sweep_iter(3, record=True)
    spins, tal = c.get_state(0)
    ts = c.get_timeseries(0)
    H = c.get_hist(0)
    assert int(H.sum()) == 3 * W
    assert np.array_equal(H, np.bincount(ts[:, 1, :].ravel(), minlength=L ** 3 + 1))
    for w in (0, 1, 1001, 2047, W - 1):
        ref = oracle.muca_run(L, d["T"], 1, d["seed"], 0, 0, n_meas=3, walker_id0=w, bonds=J)
        assert np.array_equal(spins[w], ref["spins"][0]), w
        assert np.array_equal(tal[w], ref["tallies"][0]), w
        assert np.array_equal(ts[:, :, w], ref["ts"][0]), w
    c.close()
