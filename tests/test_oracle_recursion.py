"""Pins of the oracle's weight-iteration variants (Sec. II and the recursion
of the multicanonical method it cites): the accumulated, error-weighted
recursion (reading R13 of the oracle) and the histogram flatness that the
iterate-until-flat loop stops on.  All run on the CPU.

The recursion is pinned by properties that hold whatever its implementation:
its first step from empty statistics is the plain recursion's step, a flat
histogram is its fixed point, after several iterations every neighbour ratio
is the inverse-variance weighted mean of the per-iteration estimates (written
here as a mean, not as the oracle's running update), its rule for empty bins,
and its convergence to the exact E_Delta marginal at L = 2.
"""
import numpy as np

import exact
import oracle


def plain_step(H, lnW):
    out = lnW.copy()
    oracle.update_lnW(H, out)
    return out


def test_first_step_is_the_plain_step():
    rng = np.random.default_rng(11)
    nE = 97
    H = rng.integers(0, 500, nE).astype(np.uint64)
    H[::5] = 0
    H[40:46] = 0
    lnW = rng.normal(0.0, 3.0, nE)
    got = lnW.copy()
    acc = np.zeros(nE - 1)
    oracle.update_lnW_acc(H, got, acc)
    want = plain_step(H, lnW)
    np.testing.assert_allclose(got - got[0], want - want[0], rtol=0, atol=1e-10)
    # the pair weights are H(E) H(E+1) / (H(E) + H(E+1)) where both bins were hit
    h = H.astype(float)
    both = (H[:-1] > 0) & (H[1:] > 0)
    p = np.where(both, h[:-1] * h[1:] / np.where(both, h[:-1] + h[1:], 1.0), 0.0)
    np.testing.assert_allclose(acc, p, rtol=1e-15)


def test_flat_histogram_is_a_fixed_point():
    rng = np.random.default_rng(12)
    nE = 64
    lnW = np.cumsum(rng.normal(0.0, 1.0, nE))
    acc = rng.uniform(1.0, 50.0, nE - 1)
    got = lnW.copy()
    oracle.update_lnW_acc(np.full(nE, 37, dtype=np.uint64), got, acc)
    np.testing.assert_allclose(got, lnW, rtol=0, atol=1e-12)


def test_ratios_are_the_weighted_mean_of_the_estimates():
    """Iteration m sees ratios r_m and histogram H_m and estimates
    est_m = r_m + ln H_m(E) - ln H_m(E+1) with variance 1 / p_m; after n
    iterations r = sum_m p_m est_m / sum_m p_m."""
    rng = np.random.default_rng(13)
    nE, n = 40, 5
    lnW = np.cumsum(rng.normal(0.0, 0.5, nE))
    acc = np.zeros(nE - 1)
    ests, ps = [], []
    for _ in range(n):
        H = rng.integers(1, 2000, nE).astype(np.uint64)
        h = H.astype(float)
        r = np.diff(lnW)
        ests.append(r + np.log(h[:-1]) - np.log(h[1:]))
        ps.append(h[:-1] * h[1:] / (h[:-1] + h[1:]))
        oracle.update_lnW_acc(H, lnW, acc)
        want = np.sum(np.array(ps) * np.array(ests), axis=0) / np.sum(ps, axis=0)
        np.testing.assert_allclose(np.diff(lnW), want, rtol=0, atol=1e-11)
    np.testing.assert_allclose(acc, np.sum(ps, axis=0), rtol=1e-14)


def test_empty_bins():
    """A pair with an empty bin takes the plain step (the empty bin counted as
    1) and adds nothing to its accumulated weight, whatever that weight is."""
    lnW = np.array([0.0, 0.3, -0.2, 0.5, 1.0, 0.7])
    acc = np.array([0.0, 0.0, 0.0, 4.0, 4.0])
    H = np.array([8, 0, 0, 5, 0, 3], dtype=np.uint64)
    r0 = np.diff(lnW)
    got = lnW.copy()
    a = acc.copy()
    oracle.update_lnW_acc(H, got, a)
    r = np.diff(got)
    assert abs(r[0] - (r0[0] + np.log(8.0))) < 1e-14      # frontier: plain step
    assert abs(r[1] - r0[1]) < 1e-14                      # both empty: unchanged
    assert abs(r[2] - (r0[2] - np.log(5.0))) < 1e-14      # frontier: plain step
    assert abs(r[3] - (r0[3] + np.log(5.0))) < 1e-14      # with earlier estimates too
    assert abs(r[4] - (r0[4] - np.log(3.0))) < 1e-14
    np.testing.assert_array_equal(a, acc)
    assert got[0] == lnW[0]


def test_accumulated_recursion_reaches_a_steadier_flat_histogram_l4():
    """L = 4: both recursions reach min H / mean H >= 0.5 within 40
    iterations from lnW = 0; over the last five iterations the accumulated one,
    which averages the estimates instead of following the last histogram, keeps
    the histogram flatter and steadier."""
    tail = {}
    for rec in (0, 1):
        out = oracle.muca_run(4, 1.4182, 64, 21, 40, 100, recursion=rec, want_spins=False)
        f = np.array([oracle.flatness(h)[0] for h in out["hist"]])
        assert (f >= 0.5).any()
        tail[rec] = f[-5:]
    assert tail[1].min() > tail[0].min() and tail[1].std() < tail[0].std(), tail


def exact_target(L, T):
    V = L ** 3
    probs = exact.joint_distribution(L, 1.0 / T, np.zeros(V + 1))
    g = np.zeros(V + 1)
    for (_, ed), p in probs.items():
        g[ed] += p
    return -np.log(g) + np.log(g[0])


def test_accumulated_recursion_converges_to_the_exact_marginal_l2():
    """L = 2, T = 2: the fixed point of both recursions is lnW = -ln g(E_Delta)
    up to a constant; averaging the iterations' estimates brings the
    accumulated one closer to it than the plain one, whose weights carry the
    noise of the last histogram."""
    L, T = 2, 2.0
    target = exact_target(L, T)
    err = {}
    for rec in (0, 1):
        out = oracle.muca_run(L, T, 64, 5, n_iter=14, sweeps_per_iter=400, recursion=rec)
        assert (out["hist"].sum(axis=1) == 64 * 400).all()
        got = out["lnW"] - out["lnW"][0]
        err[rec] = np.abs(got - target).max()
    assert err[1] < 0.03 and err[1] < err[0], err


def test_run_with_the_accumulated_recursion_equals_stepwise_updates():
    """The run's iterations use the accumulated update on each merged histogram."""
    L, T, W, it, sw = 2, 1.4182, 16, 4, 30
    out = oracle.muca_run(L, T, W, 9, n_iter=it, sweeps_per_iter=sw, recursion=1)
    lnW = np.zeros(L ** 3 + 1)
    acc = np.zeros(L ** 3)
    for n in range(it):
        oracle.update_lnW_acc(out["hist"][n], lnW, acc)
    np.testing.assert_array_equal(out["lnW"], lnW)
    np.testing.assert_array_equal(out["acc"], acc)


def test_flatness():
    np.testing.assert_array_equal(oracle.flatness(np.array([4, 4, 4, 4])), [1.0, 1.0, 4.0])
    np.testing.assert_allclose(oracle.flatness(np.array([2, 6, 4, 0])), [0.0, 2.0, 3.0])
    np.testing.assert_allclose(oracle.flatness(np.array([3, 6, 9])), [0.5, 1.5, 3.0])
    np.testing.assert_array_equal(oracle.flatness(np.zeros(5, dtype=np.uint64)), [0, 0, 0])
