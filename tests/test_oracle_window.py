"""Pins of the oracle's adaptive E_Delta window (reading R15 of the oracle):
the walkers move in an active window that grows after every iteration whose
merged histogram is flat over it.  All run on the CPU.

What fixes the reading independently of the code:
- a window that never grows is the fixed window of R4, which the oracle
  already runs as [e_min, e_max] with its own table and weight arrays;
- inside a window the sampler's stationary law is the exact L = 2 ensemble
  exp(-beta E_J) W(E_Delta) restricted to the window (enumeration of 3^8
  states);
- no walker is ever outside the window, so every histogram entry outside it
  is zero and every sweep of every walker is counted inside it;
- from the walkers' initial range the window reaches the exact support
  [0, V] of E_Delta, and the weights then converge to -ln of the exact
  E_Delta marginal, the fixed point of the recursion.
"""
import numpy as np
import pytest

import exact
import oracle

P_MIN = 1e-4


def initial_range(L, seed, n_walkers, walker_id0=0):
    e = [int(oracle.energies(L, oracle.init_spins(L, seed, walker_id0 + w))[1])
         for w in range(n_walkers)]
    return min(e), max(e)


def windows_before(out, window):
    """The window each iteration ran in: the initial one, then the window
    after each earlier iteration."""
    w = [tuple(window)] + [tuple(x) for x in out["windows"][:-1]]
    return np.array(w)


@pytest.mark.parametrize("grow_flat", [0.0, 1.5])
@pytest.mark.parametrize("recursion", [0, 1])
def test_a_window_that_never_grows_is_the_fixed_window(grow_flat, recursion):
    """grow_flat = 0 (off) or 1.5 (min H / mean H never exceeds 1): the run in
    the active window [a, b] of [0, V] equals the run whose whole range is
    [a, b], bin for bin, and the weights outside [a, b] stay at their start."""
    L, T, W, seed = 3, 1.4182, 24, 11
    V = L ** 3
    a, b = initial_range(L, seed, W)
    a, b = a - 2, b + 1
    lnW0 = np.random.default_rng(2).normal(0, 0.3, V + 1)
    acc0 = np.zeros(V)
    win = oracle.muca_run(L, T, W, seed, 5, 40, n_meas=7, lnW=lnW0, recursion=recursion,
                          acc=acc0, window=(a, b), grow_flat=grow_flat, grow_step=3)
    fix = oracle.muca_run(L, T, W, seed, 5, 40, n_meas=7, e_min=a, e_max=b,
                          lnW=lnW0[a:b + 1], recursion=recursion)
    assert (win["windows"] == [a, b]).all()
    np.testing.assert_array_equal(win["hist"][:, a:b + 1], fix["hist"])
    assert (win["hist"][:, :a] == 0).all() and (win["hist"][:, b + 1:] == 0).all()
    np.testing.assert_array_equal(win["spins"], fix["spins"])
    np.testing.assert_array_equal(win["tallies"], fix["tallies"])
    np.testing.assert_array_equal(win["ts"], fix["ts"])
    if recursion == 0:
        # the plain recursion moves only bins that were hit
        np.testing.assert_array_equal(win["lnW"][a:b + 1], fix["lnW"])
        np.testing.assert_array_equal(win["lnW"][:a], lnW0[:a])
        np.testing.assert_array_equal(win["lnW"][b + 1:], lnW0[b + 1:])
    else:
        # ratios inside the window are those of the fixed run (summed up from
        # bin 0 of the whole range instead of bin a: equal up to rounding)
        np.testing.assert_allclose(np.diff(win["lnW"][a:b + 1]), np.diff(fix["lnW"]),
                                   rtol=0, atol=1e-12)


@pytest.mark.parametrize("window", [(3, 6), (0, 2), (5, 8)])
def test_sampling_inside_a_window_is_the_restricted_exact_ensemble_l2(window):
    """L = 2 under fixed rough weights: final states of independent walkers
    confined to the window follow exp(-beta E_J) W(E_Delta) restricted to it
    (chi-square against the enumeration); the same weights read one bin off
    are rejected."""
    L, V, T = 2, 8, 1.0
    beta = 1.0 / T
    a, b = window
    # weights rough enough to matter, mild enough that a walker crosses a
    # window of three bins (every path passes its middle bin) in the sweeps run
    lnW = np.random.default_rng(3).normal(0, 0.7, V + 1)
    # start the walkers inside the window: all-zero spins and a few set
    n = 5000
    fin = []
    for w in range(n):
        s = np.zeros(V, dtype=np.int8)
        k = (a + b) // 2
        s[:k] = np.where(np.arange(k) % 2 == 0, 1, -1)
        tal = oracle.energies(L, s).astype(np.int32)
        thr = oracle.build_table(L, T, a, b, lnW[a:b + 1])
        oracle.sweeps(L, a, b, thr, 17, w, 0, 300, s, tal, check=True)
        fin.append((int(tal[0]), int(tal[1])))
    def restricted(lw):
        p = exact.joint_distribution(L, beta, lw)
        return {k: v for k, v in p.items() if a <= k[1] <= b}

    ok = restricted(lnW)
    z = sum(ok.values())
    ok = {k: v / z for k, v in ok.items()}
    _, _, p = exact.chi2_test(fin, ok)
    assert p > P_MIN, p
    # a slice of the weights off by one bin (lnW[E - 1], or lnW[E + 1] at the
    # lower end of the range)
    shifted = np.full(V + 1, -1e3)
    shifted[a:b + 1] = lnW[a - 1:b] if a > 0 else lnW[a + 1:b + 2]
    bad = restricted(shifted)
    zb = sum(bad.values())
    bad = {k: v / zb for k, v in bad.items()}
    _, _, pb = exact.chi2_test(fin, bad)
    assert pb < 1e-12, pb


@pytest.mark.parametrize("recursion", [0, 1])
@pytest.mark.parametrize("L,T,step,n_iter", [(2, 2.0, 1, 40), (3, 1.4182, 2, 40),
                                              (4, 1.0, 4, 240)])
def test_the_window_grows_from_the_walkers_to_the_exact_support(L, T, step, n_iter, recursion):
    """From the walkers' initial E_Delta range, with grow_flat = 0.5: every
    iteration's histogram lies inside the window it ran in and counts every
    sweep of every walker; the window never shrinks, grows by at most step
    bins a side and only after an iteration whose histogram was flat over it
    (checked with the test's own flatness); it reaches [0, V]."""
    V = L ** 3
    W, seed, sweeps = 32, 4 + L, 60
    win0 = initial_range(L, seed, W)
    assert win0 != (0, V)
    out = oracle.muca_run(L, T, W, seed, n_iter, sweeps, window=win0, grow_flat=0.5,
                          grow_step=step, recursion=recursion, want_spins=False)
    ran = windows_before(out, win0)
    for it in range(n_iter):
        lo, hi = ran[it]
        h = out["hist"][it]
        assert (h[:lo] == 0).all() and (h[hi + 1:] == 0).all(), it
        assert int(h.sum()) == W * sweeps, it
        nlo, nhi = out["windows"][it]
        assert nlo <= lo and nhi >= hi and lo - nlo <= step and nhi - hi <= step, it
        flat = oracle.flatness(h[lo:hi + 1])[0]
        grew = (nlo, nhi) != (lo, hi)
        assert grew == (flat >= 0.5 and (lo > 0 or hi < V)), (it, flat)
    assert tuple(out["windows"][-1]) == (0, V), out["windows"]


def test_new_bins_start_from_the_edge_weight():
    """At a growth step the new bins take the weight of the old edge next to
    them, and the accumulated pair weights of the pairs that contain a new bin
    are 0."""
    L, T, W, seed, sweeps = 3, 1.4182, 32, 9, 60
    V = L ** 3
    win0 = initial_range(L, seed, W)
    full = oracle.muca_run(L, T, W, seed, 30, sweeps, window=win0, grow_flat=0.5, grow_step=2,
                           recursion=1, want_spins=False)
    ran = windows_before(full, win0)
    grows = [it for it in range(30) if tuple(full["windows"][it]) != tuple(ran[it])]
    assert grows
    it = grows[0]
    out = oracle.muca_run(L, T, W, seed, it + 1, sweeps, window=win0, grow_flat=0.5,
                          grow_step=2, recursion=1, want_spins=False)
    lo, hi = ran[it]
    nlo, nhi = out["windows"][-1]
    assert (out["lnW"][nlo:lo] == out["lnW"][lo]).all()
    assert (out["lnW"][hi + 1:nhi + 1] == out["lnW"][hi]).all()
    assert (out["acc"][nlo:lo] == 0).all() and (out["acc"][hi:nhi] == 0).all()
    assert (out["acc"][lo:hi] > 0).any()
    assert nlo < lo or nhi > hi
    assert 0 <= nlo and nhi <= V


@pytest.mark.parametrize("recursion", [0, 1])
def test_grown_window_converges_to_the_exact_marginal_l2(recursion):
    """L = 2, T = 2, started from the walkers' range: once the window is
    [0, V] the weights converge to lnW = -ln g(E_Delta) up to a constant, g
    the exact marginal (the fixed point of both recursions)."""
    L, T, W, seed = 2, 2.0, 64, 5
    V = L ** 3
    win0 = initial_range(L, seed, W)
    out = oracle.muca_run(L, T, W, seed, 24, 400, window=win0, grow_flat=0.5, grow_step=1,
                          recursion=recursion, want_spins=False)
    assert tuple(out["windows"][-1]) == (0, V)
    probs = exact.joint_distribution(L, 1.0 / T, np.zeros(V + 1))
    g = np.zeros(V + 1)
    for (_, ed), p in probs.items():
        g[ed] += p
    target = -np.log(g) + np.log(g[0])
    got = out["lnW"] - out["lnW"][0]
    assert np.abs(got - target).max() < 0.25, (got, target)


def test_window_arguments():
    with pytest.raises(oracle.OracleError):
        oracle.muca_run(2, 1.0, 4, 1, 1, 1, window=(3, 2))
    with pytest.raises(oracle.OracleError):
        oracle.muca_run(2, 1.0, 4, 1, 1, 1, window=(0, 9))
    with pytest.raises(oracle.OracleError):
        oracle.muca_run(2, 1.0, 4, 1, 1, 1, window=(0, 8), grow_flat=0.5, grow_step=0)
    lo, hi = initial_range(2, 1, 4)
    with pytest.raises(oracle.OracleError):  # a walker outside the window
        oracle.muca_run(2, 1.0, 4, 1, 1, 1, window=(lo + 1, max(hi, lo + 1)))
