"""GPU runs with the weight-iteration variants against the CPU oracle (bit for
bit): the accumulated, error-weighted recursion in the plain and the graph
form, iteration until the histogram is flat (the iteration count, the
weights and the flatness record), and checkpoints that carry the recursion.
"""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def muca():
    from paper_1502_07214_gb300 import muca as m

    return m


@pytest.mark.parametrize("use_graph", [False, True])
def test_accumulated_recursion_bit_exact(use_graph):
    L, T, W, seed, n_iter, sweeps = 8, 2.0, 64, 3, 6, 50
    m = muca()
    c = m.Context([{"L": L, "T": T, "n_walkers": W}], seed=seed)
    c.set_recursion(m.REC_ACCUMULATED)
    hists = []
    if use_graph:
        c.run_graph(n_iter, sweeps)
    else:
        for _ in range(n_iter):
            c.sweep_iter(sweeps)
            hists.append(c.get_hist(0))
            c.merge_update()
    spins, tal = c.get_state(0)
    lnW, flat = c.get_lnW(0), c.get_flatness(0)
    c.close()
    ref = oracle.muca_run(L, T, W, seed, n_iter, sweeps, recursion=1)
    if not use_graph:
        np.testing.assert_array_equal(np.array(hists), ref["hist"])
    np.testing.assert_array_equal(lnW, ref["lnW"])
    np.testing.assert_array_equal(spins, ref["spins"])
    np.testing.assert_array_equal(tal, ref["tallies"])
    np.testing.assert_array_equal(flat, oracle.flatness(ref["hist"][-1]))


@pytest.mark.parametrize("rec", [0, 1])
def test_iterate_until_flat(rec):
    """L = 4, T = 1.4182, 64 walkers, 100 sweeps per iteration: the loop stops
    at the first iteration whose merged histogram has min H / mean H >= 0.5,
    the one the oracle's run reaches first."""
    L, T, W, seed, sweeps, flat_min, max_it = 4, 1.4182, 64, 21, 100, 0.5, 40
    ref = oracle.muca_run(L, T, W, seed, max_it, sweeps, recursion=rec, want_spins=False)
    f = [oracle.flatness(h)[0] for h in ref["hist"]]
    want = next(i + 1 for i, x in enumerate(f) if x >= flat_min)
    assert want < max_it
    m = muca()
    c = m.Context([{"L": L, "T": T, "n_walkers": W}], seed=seed)
    c.set_recursion(rec)
    n = c.iterate(max_it, sweeps, flat_min)
    lnW, flat = c.get_lnW(0), c.get_flatness(0)
    c.close()
    assert n == want
    np.testing.assert_array_equal(flat, oracle.flatness(ref["hist"][want - 1]))
    ref_n = oracle.muca_run(L, T, W, seed, want, sweeps, recursion=rec, want_spins=False)
    np.testing.assert_array_equal(lnW, ref_n["lnW"])


def _head(b):
    import ctypes

    assert b[:8] == b"MUCABC05"
    return 8 + 4 + 8 + 4 + ctypes.sizeof(muca().Group)  # magic, seed, sweep, n_groups, group


# one group's records after the header in format 05: recursion (int32), shard
# (2 x int32), window (3 x int32 + FP64), couplings (int32 jmax = 0: none)
REC, SHARD, WIN, BONDS = 4, 8, 20, 4
ALL = REC + SHARD + WIN + BONDS


def checkpoint_v01(src, dst, n_e):
    """The same checkpoint in the earliest format (one group): magic 01, no
    recursion field, no shard or window record, no accumulated pair weights."""
    b = open(src, "rb").read()
    head = _head(b)
    rest = b[head + ALL:]  # without the recursion, shard, window and coupling records
    lnw = rest[:8 * n_e]
    rest = rest[8 * n_e + 8 * max(n_e - 1, 1):]  # without acc
    open(dst, "wb").write(b"MUCABC01" + b[8:head] + lnw + rest)


def checkpoint_v02(src, dst):
    """The same checkpoint in format 02 (one group): no shard, window or
    coupling record."""
    b = open(src, "rb").read()
    head = _head(b)
    open(dst, "wb").write(b"MUCABC02" + b[8:head + REC] + b[head + ALL:])


def checkpoint_v03(src, dst):
    """The same checkpoint in format 03 (one group): no window or coupling
    record."""
    b = open(src, "rb").read()
    head = _head(b)
    open(dst, "wb").write(b"MUCABC03" + b[8:head + REC + SHARD] + b[head + ALL:])


def checkpoint_v04(src, dst):
    """The same checkpoint in format 04 (one group): no coupling record."""
    b = open(src, "rb").read()
    head = _head(b)
    open(dst, "wb").write(b"MUCABC04" + b[8:head + REC + SHARD + WIN] + b[head + ALL:])


def test_checkpoint_carries_the_recursion(tmp_path):
    L, T, W, seed = 8, 2.0, 40, 5
    m = muca()
    g = [{"L": L, "T": T, "n_walkers": W}]
    a = m.Context(g, seed=seed)
    a.set_recursion(m.REC_ACCUMULATED)
    for _ in range(2):
        a.sweep_iter(30)
        a.merge_update()
    path = str(tmp_path / "acc.ckpt")
    a.checkpoint(path)
    for _ in range(2):
        a.sweep_iter(30)
        a.merge_update()
    want_lnW, want_spins = a.get_lnW(0), a.get_state(0)[0]
    a.close()
    b = m.Context(g, seed=seed)  # plain recursion until the restore
    b.restore(path)
    for _ in range(2):
        b.sweep_iter(30)
        b.merge_update()
    np.testing.assert_array_equal(b.get_lnW(0), want_lnW)
    np.testing.assert_array_equal(b.get_state(0)[0], want_spins)
    b.close()
    # the earlier format restores with the plain recursion
    c = m.Context(g, seed=seed)
    c.restore(path)
    c.set_recursion(m.REC_PLAIN)
    for _ in range(2):
        c.sweep_iter(30)
        c.merge_update()
    plain_lnW = c.get_lnW(0)
    c.close()
    old = str(tmp_path / "acc01.ckpt")
    checkpoint_v01(path, old, L ** 3 + 1)
    d = m.Context(g, seed=seed)
    d.set_recursion(m.REC_ACCUMULATED)
    d.restore(old)
    for _ in range(2):
        d.sweep_iter(30)
        d.merge_update()
    np.testing.assert_array_equal(d.get_lnW(0), plain_lnW)
    d.close()
    # formats 02 (no shard record: every walker of the group), 03 (no window
    # record: the fixed window [e_min, e_max]) and 04 (no couplings: the clean
    # model) restore the run
    for name, conv in (("acc02.ckpt", checkpoint_v02), ("acc03.ckpt", checkpoint_v03),
                       ("acc04.ckpt", checkpoint_v04)):
        v = str(tmp_path / name)
        conv(path, v)
        e = m.Context(g, seed=seed)
        e.restore(v)
        assert e.get_window(0) == (0, L ** 3)
        for _ in range(2):
            e.sweep_iter(30)
            e.merge_update()
        np.testing.assert_array_equal(e.get_lnW(0), want_lnW)
        np.testing.assert_array_equal(e.get_state(0)[0], want_spins)
        e.close()


def test_recursion_errors():
    m = muca()
    c = m.Context([{"L": 4, "T": 1.0, "n_walkers": 8}], seed=1)
    np.testing.assert_array_equal(c.get_flatness(0), np.zeros(3))
    with pytest.raises(m.MucaError) as e:
        c.set_recursion(2)
    assert e.value.code == m.ERR_INVALID_ARG
    with pytest.raises(m.MucaError) as e:
        c.iterate(3, 0, 0.5)
    assert e.value.code == m.ERR_INVALID_ARG
    with pytest.raises(m.MucaError) as e:
        c.get_flatness(1)
    assert e.value.code == m.ERR_INVALID_ARG
    assert c.iterate(0, 10, 0.5) == 0
    c.close()
