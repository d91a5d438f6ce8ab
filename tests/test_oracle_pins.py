"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test ties one part of the oracle to something other than itself:
published known-answer vectors, closed-form energies, exact enumeration of
the L = 2 lattice (3^8 states), the Ising limit Delta -> -inf (Sec. I), the
canonical special case of the weights and the two-ground-state switch at
Delta_0 = zJ/2 = 3 (Sec. I).  All run on the CPU.
"""
import os

import numpy as np
import pytest

import exact
import oracle
from paper_1502_07214_gb300 import workloads as wl

HERE = os.path.dirname(os.path.abspath(__file__))
P_MIN = 1e-4  # fixed in advance for every chi-square test below


def read_kat():
    rows = []
    with open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            rows.append([int(x, 16) for x in line.split()])
    return rows


def test_philox_known_answers():
    rows = read_kat()
    assert len(rows) == 3
    for r in rows:
        assert list(oracle.philox(r[0:4], r[4:6])) == r[6:10]


# --------------------------------------------------------------------------
# Energies (Eq. 1) on configurations with closed-form values.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("L", [2, 3, 4, 5, 8])
def test_energies_closed_forms(L):
    V = L ** 3
    one = np.ones(V, dtype=np.int8)
    assert list(oracle.energies(L, one)) == [-3 * V, V, V]
    assert list(oracle.energies(L, -one)) == [-3 * V, V, -V]
    assert list(oracle.energies(L, 0 * one)) == [0, 0, 0]
    single = np.zeros(V, dtype=np.int8)
    single[V // 2] = 1
    assert list(oracle.energies(L, single)) == [0, 1, 1]
    # a pair along x: one bond for L >= 3, both bonds of the pair at L = 2
    pair = np.zeros(V, dtype=np.int8)
    pair[0] = 1
    pair[1] = -1
    assert list(oracle.energies(L, pair)) == [2 if L == 2 else 1, 2, 0]
    if L % 2 == 0:
        x, y, z = np.meshgrid(np.arange(L), np.arange(L), np.arange(L), indexing="ij")
        # site i = x + L (y + L z): build in (z, y, x) order
        par = (x + y + z) % 2
        chk = np.where(par == 0, 1, -1).astype(np.int8).transpose(2, 1, 0).ravel()
        assert list(oracle.energies(L, chk)) == [3 * V, V, 0]


def test_energies_brute_force_l2():
    st = exact.all_states(2)[::7]
    ej, ed, m = exact.state_energies(st, 2)
    for k in range(len(st)):
        e = oracle.energies(2, st[k].astype(np.int8))
        assert (e[0], e[1], e[2]) == (ej[k], ed[k], m[k])


def test_init_spins_uniform():
    from scipy import stats

    L = 8
    s = np.concatenate([oracle.init_spins(L, 11, w) for w in range(64)])
    assert set(np.unique(s)) <= {-1, 0, 1}
    counts = np.array([(s == v).sum() for v in (-1, 0, 1)])
    chi2 = ((counts - len(s) / 3) ** 2 / (len(s) / 3)).sum()
    assert stats.chi2.sf(chi2, 2) > P_MIN
    # different walkers and seeds give different streams
    assert not np.array_equal(oracle.init_spins(L, 11, 0), oracle.init_spins(L, 11, 1))
    assert not np.array_equal(oracle.init_spins(L, 11, 0), oracle.init_spins(L, 12, 0))


# --------------------------------------------------------------------------
# Acceptance table properties (reading R4).
# --------------------------------------------------------------------------
def test_table_structure():
    L, T = 3, 1.3
    V = L ** 3
    rng = np.random.default_rng(5)
    lnW = np.cumsum(rng.normal(0, 0.7, V + 1))
    thr = oracle.build_table(L, T, 0, V, lnW)
    assert thr.shape == (V + 1, 3, 25)
    assert thr.max() <= 2 ** 31
    # leaving the window is never accepted
    assert (thr[0, 0, :] == 0).all() and (thr[V, 2, :] == 0).all()
    # d = 0 does not depend on E_Delta, and is 2^31 exactly for dE_J <= 0
    assert (thr[:, 1, :] == thr[0, 1, :]).all()
    assert (thr[0, 1, :13] == 2 ** 31).all() and (thr[0, 1, 13:] < 2 ** 31).all()
    # non-increasing in dE_J for every (E, d) inside the window
    inner = thr[1:V, :, :].astype(np.int64)
    assert (np.diff(inner, axis=2) <= 0).all()
    # shifting lnW by a constant changes nothing
    assert np.array_equal(oracle.build_table(L, T, 0, V, lnW + 123.25), thr)


# --------------------------------------------------------------------------
# Sampler against exact enumeration of L = 2 (3^8 = 6561 states).
# --------------------------------------------------------------------------
def independent_final_states(L, T, lnW, n_walkers, n_sweeps, seed):
    out = oracle.muca_run(L, T, n_walkers, seed, n_iter=0, sweeps_per_iter=0, n_meas=n_sweeps,
                          lnW=lnW, check=True)
    ts = out["ts"]
    return ts[:, -1, :]  # one sample per walker: independent across walkers


@pytest.mark.parametrize("case", ["flat", "canonical", "rough"])
def test_sampler_exact_enumeration_l2(case):
    L, V = 2, 8
    T = {"flat": 2.0, "canonical": 1.4182, "rough": 1.0}[case]
    beta = 1.0 / T
    E = np.arange(V + 1)
    if case == "flat":
        lnW = np.zeros(V + 1)
    elif case == "canonical":
        lnW = -beta * 2.8 * E  # a canonical run at Delta = 2.8
    else:
        lnW = np.random.default_rng(3).normal(0, 1.5, V + 1)
    probs = exact.joint_distribution(L, beta, lnW)
    fin = independent_final_states(L, T, lnW, n_walkers=20000, n_sweeps=24, seed=7)
    keys = [(int(a), int(b)) for a, b, _ in fin]
    chi2, dof, p = exact.chi2_test(keys, probs)
    assert p > P_MIN, (chi2, dof, p)


def test_sampler_detects_planted_sign_error():
    """The enumeration test has power: the distribution with the opposite sign of
    E_J (what a flipped dE_J would sample) fails it."""
    L, V, T = 2, 8, 2.0
    beta = 1.0 / T
    lnW = np.zeros(V + 1)
    wrong = exact.joint_distribution(L, -beta, lnW)
    fin = independent_final_states(L, T, lnW, n_walkers=20000, n_sweeps=24, seed=7)
    keys = [(int(a), int(b)) for a, b, _ in fin]
    keys = [k for k in keys if k in wrong]
    _, _, p = exact.chi2_test(keys, wrong)
    assert p < 1e-12


def test_ising_limit_l2():
    """Delta -> -inf (Sec. I): with lnW = -beta Delta E_Delta, Delta = -1e6, no
    vacancy is ever created from an all-(+-1) state, and E_J follows the exact
    Ising distribution on 2^8 states."""
    L, V, T = 2, 8, 1.8
    beta = 1.0 / T
    lnW = -beta * (-1e6) * np.arange(V + 1)
    thr = oracle.build_table(L, T, 0, V, lnW)
    assert (thr[1:, 0, :] == 0).all()
    rng = np.random.default_rng(1)
    keys = []
    for w in range(6000):
        s = rng.choice(np.array([-1, 1], dtype=np.int8), size=V)
        tal = oracle.energies(L, s).astype(np.int32)
        ts = oracle.sweeps(L, 0, V, thr, 9, w, 0, 20, s, tal, record=True, check=True)
        assert (ts[:, 1] == V).all()
        keys.append((int(ts[-1, 0]), V))
    probs = exact.joint_distribution(L, beta, np.zeros(V + 1), values=(-1, 1))
    probs = {k: p for k, p in probs.items()}
    _, _, p = exact.chi2_test(keys, probs)
    assert p > P_MIN


@pytest.mark.parametrize("L,T", [(3, 2.0), (4, 0.9), (5, 1.4182)])
def test_running_tallies_equal_recomputed(L, T):
    V = L ** 3
    lnW = np.random.default_rng(L).normal(0, 2.0, V + 1)
    out = oracle.muca_run(L, T, 6, 3, n_iter=2, sweeps_per_iter=5, n_meas=5, lnW=lnW,
                          check=True)
    for w in range(6):
        e = oracle.energies(L, out["spins"][w])
        assert list(e) == list(out["tallies"][w])
        assert -3 * V <= e[0] <= 3 * V and 0 <= e[1] <= V and abs(e[2]) <= e[1]


def test_window_is_respected():
    L, T = 4, 1.0
    V = L ** 3
    thr_lo, thr_hi = 30, 50
    lnW = np.zeros(thr_hi - thr_lo + 1)
    thr = oracle.build_table(L, T, thr_lo, thr_hi, lnW)
    rng = np.random.default_rng(0)
    s = np.zeros(V, dtype=np.int8)
    s[rng.choice(V, 40, replace=False)] = 1
    tal = oracle.energies(L, s).astype(np.int32)
    ts = oracle.sweeps(L, thr_lo, thr_hi, thr, 1, 0, 0, 200, s, tal, record=True, check=True)
    assert ts[:, 1].min() >= thr_lo and ts[:, 1].max() <= thr_hi
    assert ts[:, 1].min() == thr_lo or ts[:, 1].max() == thr_hi  # the walker reaches an edge


def test_histogram_total_and_flat_weights_l2():
    """Sum of the merged histogram = walkers x sweeps; after the weight
    iteration converges, lnW(E) - lnW(0) = -ln g(E) + ln g(0) with g the exact
    E_Delta marginal of exp(-beta E_J) (the fixed point of the recursion)."""
    L, V, T = 2, 8, 2.0
    beta = 1.0 / T
    out = oracle.muca_run(L, T, 64, 5, n_iter=14, sweeps_per_iter=400, lnW=np.zeros(V + 1))
    assert (out["hist"].sum(axis=1) == 64 * 400).all()
    probs = exact.joint_distribution(L, beta, np.zeros(V + 1))
    g = np.zeros(V + 1)
    for (a, b), p in probs.items():
        g[b] += p
    target = -np.log(g) + np.log(g[0])
    got = out["lnW"] - out["lnW"][0]
    assert np.abs(got - target).max() < 0.25, (got, target)
    last = out["hist"][-1].astype(float)
    assert last.min() > 0.5 * last.mean()


# --------------------------------------------------------------------------
# Reweighting (Eq. 3, Eq. 6).
# --------------------------------------------------------------------------
def test_reweight_canonical_special_case():
    """lnW = -beta Delta_0 E_Delta makes every weight equal at Delta_0: the
    reweighted values are the plain sample statistics."""
    rng = np.random.default_rng(2)
    V, T, d0 = 512, 2.0, 2.5
    beta = 1 / T
    n = 5000
    ed = rng.integers(0, V + 1, n).astype(np.int32)
    ej = (rng.integers(-3 * V, 1, n)).astype(np.int32)
    m = (rng.integers(-1, 2, n) * rng.integers(0, V // 2, n)).astype(np.int32)
    lnW = -beta * d0 * np.arange(V + 1)
    out = oracle.reweight(ej, ed, m, lnW, 0, beta, V, [d0])[0]
    ejf, edf, mf = ej.astype(float), ed.astype(float), m.astype(float) / V
    cov = np.mean(ejf * edf) - ejf.mean() * edf.mean()
    want = [ejf.mean(), edf.mean(), -beta * cov,
            beta * V * (np.mean(mf ** 2) - np.mean(np.abs(mf)) ** 2),
            1 - np.mean(mf ** 4) / (3 * np.mean(mf ** 2) ** 2)]
    np.testing.assert_allclose(out, want, rtol=1e-10)


def test_reweight_two_ground_states_switch():
    """Sec. I: at T -> 0 the all-(+-1) states (E_J = -3V, E_Delta = V) and the
    all-0 state (E = 0) exchange stability at Delta_0 = zJ/2 = 3.  A series
    holding n1 samples of the first and n0 of the second, drawn with weights
    W, reweights to <E_Delta>/V = r/(1+r), r = (n1/n0) (W0/W1) exp(-beta Delta V)."""
    V, T = 64, 0.25
    beta = 1 / T
    n1, n0 = 300, 500
    lnW = np.zeros(V + 1)
    lnW[V] = -beta * 3 * V  # W(V) makes both states equally likely at Delta = 3
    ed = np.array([V] * n1 + [0] * n0, dtype=np.int32)
    ej = np.array([-3 * V] * n1 + [0] * n0, dtype=np.int32)
    m = np.array([V, -V] * (n1 // 2) + [0] * n0, dtype=np.int32)
    grid = np.linspace(2.95, 3.05, 11)
    out = oracle.reweight(ej, ed, m, lnW, 0, beta, V, grid)
    lr = np.log(n1 / n0) + (0.0 - lnW[V]) - beta * grid * V
    r = np.exp(lr)
    np.testing.assert_allclose(out[:, 1] / V, r / (1 + r), rtol=1e-12)
    # the crossing of 1/2 sits at Delta = 3 + ln(n1/n0)/(beta V) -> 3 as T -> 0
    cross = 3 + np.log(n1 / n0) / (beta * V)
    assert abs(cross - 3) < 2e-3
    # C = -beta cov(E_J, E_Delta) with E_J = -3 E_Delta on this series
    q = r / (1 + r)
    np.testing.assert_allclose(out[:, 2], -beta * (-3) * V * V * q * (1 - q), rtol=1e-9)


def test_exact_l2_switch_at_low_temperature():
    """Sec. I: as T -> 0 the ordered (all +1 or all -1) and the empty (all 0)
    ground states exchange at Delta_0 = zJ/2 = 3.  Exact enumeration of L = 2
    (3^8 states) at T = 0.05: <E_Delta>/V crosses 1/2 at 3 + T ln 2 / V, the
    two ordered states against the one empty state; every excited state is
    suppressed by at least exp(-3/T).  Pins the model reading (Eq. 1, R1) that
    the sampler pins rest on."""
    L, T = 2, 0.05
    V, beta = L ** 3, 1.0 / T
    E = np.arange(V + 1)

    def e_delta(delta):
        P = exact.joint_distribution(L, beta, -beta * delta * E)
        return sum(p * ed for (_, ed), p in P.items()) / V

    lo, hi = 2.9, 3.1
    assert e_delta(lo) > 0.5 > e_delta(hi)
    for _ in range(60):
        mid = lo + (hi - lo) / 2
        if e_delta(mid) > 0.5:
            lo = mid
        else:
            hi = mid
    assert abs(lo - (3 + T * np.log(2) / V)) < 1e-9
    assert abs(lo - 3) < T


def test_reweight_sampler_against_exact_l2():
    """Sampler + reweighting together against exact canonical averages at L = 2
    over a Delta range (Eq. 2, Eq. 3, Eq. 6)."""
    L, V, T = 2, 8, 1.4182
    beta = 1 / T
    # weights close to the converged MUCA weights so every E_Delta is visited
    probs = exact.joint_distribution(L, beta, np.zeros(V + 1))
    g = np.zeros(V + 1)
    for (a, b), p in probs.items():
        g[b] += p
    lnW = -np.log(g)
    nw, ns = 256, 400
    out = oracle.muca_run(L, T, nw, 21, n_iter=0, sweeps_per_iter=0, n_meas=ns, lnW=lnW)
    ts = out["ts"][:, 50:, :]
    grid = np.array([2.0, 2.6, 2.85, 3.0, 3.3])
    # error bars from 16 jackknife blocks of walkers (walkers are independent)
    full = oracle.reweight(ts[..., 0], ts[..., 1], ts[..., 2], lnW, 0, beta, V, grid)
    blocks = np.array_split(np.arange(nw), 16)
    jk = []
    for b in blocks:
        keep = np.setdiff1d(np.arange(nw), b)
        s = ts[keep]
        jk.append(oracle.reweight(s[..., 0], s[..., 1], s[..., 2], lnW, 0, beta, V, grid))
    jk = np.array(jk)
    err = np.sqrt((len(blocks) - 1) * ((jk - jk.mean(axis=0)) ** 2).mean(axis=0))
    for k, d in enumerate(grid):
        want = exact.canonical_averages(L, beta, d)
        z = np.abs(full[k] - want) / np.maximum(err[k], 1e-12)
        assert (z < 5).all(), (d, full[k], want, err[k])


def test_reweight_invariances_and_binary128():
    rng = np.random.default_rng(4)
    V, beta = 1000, 1 / 1.4182
    n = 20000
    ed = rng.integers(200, 800, n).astype(np.int32)
    ej = (-2 * ed + rng.integers(-300, 300, n)).astype(np.int32)
    m = (rng.integers(-1, 2, n) * ed).astype(np.int32)
    E = np.arange(V + 1)
    lnW = -beta * 2.8 * E + 3.0 * np.sin(E / 50.0)
    grid = np.linspace(2.75, 2.85, 5)
    a = oracle.reweight(ej, ed, m, lnW, 0, beta, V, grid)
    b = oracle.reweight(ej, ed, m, lnW + 1e4, 0, beta, V, grid)
    np.testing.assert_allclose(a, b, rtol=1e-9)
    # sample order does not matter
    p = rng.permutation(n)
    c = oracle.reweight(ej[p], ed[p], m[p], lnW, 0, beta, V, grid)
    np.testing.assert_allclose(a, c, rtol=1e-12)
    q = oracle.reweight_q(ej, ed, m, lnW, 0, beta, V, grid)
    np.testing.assert_allclose(a, q, rtol=1e-12)


def test_fp64_oracle_against_binary128_at_large_volume():
    """FP64 against binary128 on an L=32 series across the transition.  The
    bound follows from the arithmetic: the log-weight ratio of the two peaks is
    an FP64 number of size beta Delta |E1 - E2| ~ 4e4 (rounding ~1e-11), so the
    observables at the transition carry ~1e-11 relative error; away from it
    they stay near 1e-15."""
    from paper_1502_07214_gb300 import workloads as wl

    ej, ed, m, lnW, dt = wl.synthetic_series(L=32, n_walkers=64, n_samples=300, seed=5)
    beta = 1 / 1.4182
    grid = wl.delta_grid(dt, 0.05, 9)
    a = oracle.reweight(ej, ed, m, lnW, 0, beta, 32 ** 3, grid)
    q = oracle.reweight_q(ej, ed, m, lnW, 0, beta, 32 ** 3, grid)
    scale = np.maximum(np.abs(q), 1e-3 * np.abs(q).max(axis=0, keepdims=True))
    err = np.abs(a - q) / scale
    assert err.max() < 1e-10
    assert np.median(err) < 1e-14


# ---------------------------------------------------------------- Delta*_L
def _two_state_rows(V, n_rows, per_row1, per_row0):
    """Rows (sweeps) of the two T = 0 ground states: per_row1 samples of the
    all-(+-1) state (E_J = -3V, E_Delta = V) and per_row0 of the all-0 state."""
    ed = np.array([[V] * per_row1 + [0] * per_row0] * n_rows, dtype=np.int32)
    ej = np.array([[-3 * V] * per_row1 + [0] * per_row0] * n_rows, dtype=np.int32)
    return ej, ed


def test_peak_two_ground_states_closed_form():
    """Sec. III's Delta*_L on the two-state series: C = 3 beta V^2 q (1 - q) with
    q the reweighted weight of the all-(+-1) state, largest at q = 1/2, i.e. at
    Delta* = 3 + (ln(n1/n0) - lnW(V) + lnW(0)) / (beta V) - 3 = 3 + ln(n1/n0)/(beta V)
    (lnW(V) = -3 beta V), with C* = 3 beta V^2 / 4.  Every jackknife subset holds
    the same proportions, so all subsets agree and the jackknife spread is 0."""
    V, T = 64, 0.25
    beta = 1 / T
    lnW = np.zeros(V + 1)
    lnW[V] = -beta * 3 * V
    ej, ed = _two_state_rows(V, n_rows=40, per_row1=3, per_row0=5)
    out = oracle.find_peak(ej, ed, lnW, 0, beta, 2.9, 3.1, n_iter=60, n_jack=8)
    want = 3 + np.log(3 / 5) / (beta * V)
    np.testing.assert_allclose(out[:, 0], want, rtol=0, atol=1e-12)
    np.testing.assert_allclose(out[:, 1], 3 * beta * V * V / 4, rtol=1e-12)


def test_peak_subsets_are_the_series_without_their_block():
    """Subset i of the jackknife is the full-series search on the series with
    rows [i n / w, (i + 1) n / w) removed: built here by slicing, the two agree
    exactly."""
    ej, ed, m, lnW, dt = wl.synthetic_series(L=6, T=1.4182, n_walkers=16, n_samples=60, seed=21)
    beta = 1 / 1.4182
    grid = np.linspace(dt - 0.3, dt + 0.3, 121)
    c = oracle.reweight(ej, ed, m, lnW, 0, beta, 6 ** 3, grid)[:, 2]
    k = int(np.argmax(c))
    lo, hi = grid[max(k - 3, 0)], grid[min(k + 3, len(grid) - 1)]
    w = 5
    out = oracle.find_peak(ej, ed, lnW, 0, beta, lo, hi, n_iter=50, n_jack=w)
    n = ed.shape[0]
    for i in range(w):
        keep = np.r_[0:i * n // w, (i + 1) * n // w:n]
        sub = oracle.find_peak(ej[keep], ed[keep], lnW, 0, beta, lo, hi, n_iter=50)
        assert np.array_equal(out[1 + i], sub[0])


def test_peak_is_the_maximum_of_the_reweighted_c():
    """Delta* from the bisection on dC/dDelta against a dense scan of C(Delta)
    by the reweighting (Eq. 3, 6): the scan's largest value lies within one
    grid step of Delta*, and no scanned C exceeds C*."""
    ej, ed, m, lnW, dt = wl.synthetic_series(L=8, T=1.4182, n_walkers=32, n_samples=200, seed=5)
    beta, V = 1 / 1.4182, 8 ** 3
    coarse = np.linspace(dt - 0.3, dt + 0.3, 61)
    c = oracle.reweight(ej, ed, m, lnW, 0, beta, V, coarse)[:, 2]
    k = int(np.argmax(c))
    lo, hi = coarse[k - 2], coarse[k + 2]
    out = oracle.find_peak(ej, ed, lnW, 0, beta, lo, hi, n_iter=60)
    ds, cs = out[0]
    fine = np.linspace(lo, hi, 801)
    cf = oracle.reweight(ej, ed, m, lnW, 0, beta, V, fine)[:, 2]
    assert abs(fine[int(np.argmax(cf))] - ds) <= (fine[1] - fine[0])
    assert cf.max() <= cs * (1 + 1e-12)
    assert abs(oracle.reweight(ej, ed, m, lnW, 0, beta, V, [ds])[0, 2] - cs) <= 1e-12 * abs(cs)


def test_peak_rejects_an_interval_without_the_maximum():
    V, T = 64, 0.25
    beta = 1 / T
    lnW = np.zeros(V + 1)
    lnW[V] = -beta * 3 * V
    ej, ed = _two_state_rows(V, n_rows=10, per_row1=3, per_row0=5)
    with pytest.raises(oracle.OracleError):
        oracle.find_peak(ej, ed, lnW, 0, beta, 3.05, 3.2)


# ---------------------------------------------------- equal height, barrier
def _double_well(L, T, delta_t):
    """lnW and the series of the synthetic recipe with every E_Delta in [0, V]
    occupied exactly once per row: the reweighted distribution at delta_t is
    exp(0.6 L^2 (well(e) - max well)), peaks at e = 0.25 and 0.8, minimum at
    e = 0.525 (V = L^3 divisible by 40 puts all three on bins)."""
    V = L ** 3
    beta = 1.0 / T
    E = np.arange(V + 1, dtype=np.float64)
    e = E / V
    well = -((e - 0.25) * (e - 0.8)) ** 2 / 0.01
    lnW = -(beta * delta_t * E + (0.6 * L * L) * (well - well.max()))
    rows = np.array([np.roll(np.arange(V + 1), 37 * r) for r in range(8)], dtype=np.int32)
    barrier = 0.6 * L * L * (well.max() - well[int(0.525 * V)])
    return V, beta, lnW, rows, barrier


def test_equal_height_closed_form():
    L, T, dt = 10, 1.0, 2.6
    V, beta, lnW, rows, barrier = _double_well(L, T, dt)
    out = oracle.equal_height(rows, lnW, 0, beta, int(0.525 * V), dt - 0.05, dt + 0.05,
                              n_iter=60, n_jack=4)
    np.testing.assert_allclose(out[:, 0], dt, rtol=0, atol=1e-12)
    np.testing.assert_allclose(out[:, 1], barrier / (2 * beta * dt), rtol=1e-9)
    assert np.all(out[:, 2] == 0.25 * V) and np.all(out[:, 3] == 0.8 * V)
    assert np.all(out[:, 4] == 0.525 * V)
    assert np.all(out[1:] == out[1])  # identical subsets, identical results


def test_equal_height_noisy_series_near_the_construction():
    """The sampled synthetic series (Poisson noise in every bin) puts Delta_eqh
    near the constructed transition field."""
    ej, ed, m, lnW, dt = wl.synthetic_series(L=10, T=1.4182, n_walkers=64, n_samples=2000, seed=7)
    out = oracle.equal_height(ed, lnW, 0, 1 / 1.4182, 525, dt - 0.05, dt + 0.05)
    assert abs(out[0, 0] - dt) < 2e-3


def test_equal_height_rejects_an_interval_without_it():
    L, T, dt = 10, 1.0, 2.6
    V, beta, lnW, rows, barrier = _double_well(L, T, dt)
    with pytest.raises(oracle.OracleError):
        oracle.equal_height(rows, lnW, 0, beta, int(0.525 * V), dt + 0.01, dt + 0.05)
