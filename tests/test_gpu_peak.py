"""GPU Delta*_L and C*_L (Sec. III) against the CPU oracle.

The bisection takes the same decisions on both sides except where dC/dDelta
is within rounding of zero, so Delta* agrees to far below the FP64 bracket
width: tolerance 1e-9 absolute.  C* is taken at a maximum, where it is flat
in Delta: relative tolerance 1e-10.  The jackknife errors are differences of
nearly equal numbers: relative tolerance 1e-5.
"""
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()


def bracket(ej, ed, m, lnW, beta, V, centre, half=0.3, n=61, k_side=2):
    """An interval around the largest C of a coarse oracle scan."""
    grid = np.linspace(centre - half, centre + half, n)
    c = oracle.reweight(ej, ed, m, lnW, 0, beta, V, grid)[:, 2]
    k = int(np.argmax(c))
    return grid[max(k - k_side, 0)], grid[min(k + k_side, n - 1)]


def jack_err(x):
    w = len(x)
    return np.sqrt((w - 1) / w * np.sum((x - x.mean()) ** 2))


@pytest.mark.parametrize("L,nw,ns,w", [(8, 32, 200, 5), (12, 64, 150, 10), (16, 128, 400, 4)])
def test_peak_matches_oracle(L, nw, ns, w):
    T = 1.4182
    beta, V = 1 / T, L ** 3
    ej, ed, m, lnW, dt = wl.synthetic_series(L=L, T=T, n_walkers=nw, n_samples=ns, seed=L + 1)
    lo, hi = bracket(ej, ed, m, lnW, beta, V, dt)
    ref = oracle.find_peak(ej, ed, lnW, 0, beta, lo, hi, n_iter=60, n_jack=w)
    ds, de, cs, cse, sub = muca().find_peak(dev(ej), dev(ed), lnW, 0, beta, lo, hi, n_iter=60,
                                            n_jack=w)
    assert abs(ds - ref[0, 0]) <= 1e-9
    assert abs(cs - ref[0, 1]) <= 1e-10 * abs(ref[0, 1])
    np.testing.assert_allclose(sub[:, 0], ref[1:, 0], rtol=0, atol=1e-9)
    np.testing.assert_allclose(sub[:, 1], ref[1:, 1], rtol=1e-10)
    np.testing.assert_allclose(de, jack_err(ref[1:, 0]), rtol=1e-5)
    np.testing.assert_allclose(cse, jack_err(ref[1:, 1]), rtol=1e-5)


def test_peak_two_ground_states_closed_form():
    """Delta* = 3 + ln(n1/n0)/(beta V), C* = 3 beta V^2 / 4 (the oracle's pin).
    The jackknife subsets hold the same proportions, so their spread is zero up
    to rounding (the subsets' sums round differently from the full ones)."""
    V, T = 64, 0.25
    beta = 1 / T
    lnW = np.zeros(V + 1)
    lnW[V] = -beta * 3 * V
    ed = np.array([[V] * 3 + [0] * 5] * 40, dtype=np.int32)
    ej = np.array([[-3 * V] * 3 + [0] * 5] * 40, dtype=np.int32)
    ds, de, cs, cse, sub = muca().find_peak(dev(ej), dev(ed), lnW, 0, beta, 2.9, 3.1, n_jack=8)
    assert abs(ds - (3 + np.log(3 / 5) / (beta * V))) <= 1e-12
    assert abs(cs - 3 * beta * V * V / 4) <= 1e-12 * cs
    assert de <= 1e-12 and cse <= 1e-12 * cs


def test_peak_strided_rows_of_the_context_layout():
    """Rows with a stride ([sample][field][walker], as the context records them)."""
    L, T, W, S = 8, 1.4182, 24, 90
    beta, V = 1 / T, L ** 3
    ej, ed, m, lnW, dt = wl.synthetic_series(L=L, T=T, n_walkers=W, n_samples=S, seed=31)
    lo, hi = bracket(ej, ed, m, lnW, beta, V, dt)
    packed = np.stack([ej, ed, m], axis=1).astype(np.int32)  # [S][3][W]
    buf = torch.from_numpy(packed.ravel()).cuda()
    base = buf.data_ptr()
    got = muca().find_peak(base, base + 4 * W, lnW, 0, beta, lo, hi, n_jack=3, n_rows=S,
                           row_len=W, row_stride=3 * W)
    ref = oracle.find_peak(ej, ed, lnW, 0, beta, lo, hi, n_jack=3)
    assert abs(got[0] - ref[0, 0]) <= 1e-9
    np.testing.assert_allclose(got[4][:, 0], ref[1:, 0], rtol=0, atol=1e-9)


def test_peak_errors():
    V, T = 64, 0.25
    beta = 1 / T
    lnW = np.zeros(V + 1)
    lnW[V] = -beta * 3 * V
    ed = np.array([[V] * 3 + [0] * 5] * 10, dtype=np.int32)
    ej = np.array([[-3 * V] * 3 + [0] * 5] * 10, dtype=np.int32)
    with pytest.raises(muca().MucaError) as e:  # the maximum is not inside
        muca().find_peak(dev(ej), dev(ed), lnW, 0, beta, 3.05, 3.2)
    assert e.value.code == muca().ERR_INVALID_ARG
    with pytest.raises(muca().MucaError) as e:  # n_jack = 1 has no jackknife
        muca().find_peak(dev(ej), dev(ed), lnW, 0, beta, 2.9, 3.1, n_jack=1)
    assert e.value.code == muca().ERR_INVALID_ARG
    bad = ed.copy()
    bad[3, 2] = V + 7
    with pytest.raises(muca().MucaError) as e:
        muca().find_peak(dev(ej), dev(bad), lnW, 0, beta, 2.9, 3.1)
    assert e.value.code == muca().ERR_WINDOW


def test_full_size_peak_is_the_maximum_of_c():
    """The reweight workload (4096 walkers x 10^4 samples of L = 32) with 20
    jackknife blocks: C(Delta*) from the FP64 reweighting equals C*, no point
    of a fine scan around Delta* has a larger C, and the subsets' Delta* lie
    within a few jackknife errors of Delta*."""
    s = wl.REWEIGHT
    ej, ed, m, lnW, dt = wl.synthetic_series()
    beta, V = 1 / s["T"], s["L"] ** 3
    e_j, e_d, mm = dev(ej), dev(ed), dev(m)
    coarse = wl.delta_grid(dt, 0.05, 401)
    c = muca().reweight(e_j, e_d, mm, lnW, 0, beta, V, coarse, 64)[:, 2]
    k = int(np.argmax(c))
    lo, hi = coarse[k - 3], coarse[k + 3]
    ds, de, cs, cse, sub = muca().find_peak(e_j, e_d, lnW, 0, beta, lo, hi, n_jack=20)
    at = muca().reweight(e_j, e_d, mm, lnW, 0, beta, V, [ds], 64)[0, 2]
    assert abs(at - cs) <= 1e-10 * abs(cs)
    fine = np.linspace(lo, hi, 241)
    cf = muca().reweight(e_j, e_d, mm, lnW, 0, beta, V, fine, 64)[:, 2]
    assert cf.max() <= cs * (1 + 1e-12)
    assert abs(fine[int(np.argmax(cf))] - ds) <= fine[1] - fine[0]
    assert de > 0 and np.all(np.abs(sub[:, 0] - ds) <= 10 * de)


# ---------------------------------------------------- equal height, barrier
def double_well(L, T, delta_t):
    """Every E_Delta in [0, V] once per row under the synthetic recipe's lnW:
    equal peaks at e = 0.25 and 0.8 exactly at delta_t, minimum at e = 0.525."""
    V = L ** 3
    beta = 1.0 / T
    E = np.arange(V + 1, dtype=np.float64)
    e = E / V
    well = -((e - 0.25) * (e - 0.8)) ** 2 / 0.01
    lnW = -(beta * delta_t * E + (0.6 * L * L) * (well - well.max()))
    rows = np.array([np.roll(np.arange(V + 1), 37 * r) for r in range(8)], dtype=np.int32)
    return V, beta, lnW, rows, 0.6 * L * L * (well.max() - well[int(0.525 * V)])


def test_equal_height_closed_form_and_oracle():
    L, T, dt = 10, 1.0, 2.6
    V, beta, lnW, rows, barrier = double_well(L, T, dt)
    got = muca().equal_height(dev(rows), lnW, 0, beta, int(0.525 * V), dt - 0.05, dt + 0.05,
                              n_jack=4)
    assert abs(got[0] - dt) <= 1e-12
    assert abs(got[2] - barrier / (2 * beta * dt)) <= 1e-9 * got[2]
    assert got[4] == (250, 800, 525)
    assert got[1] <= 1e-12 and got[3] <= 1e-9 * got[2]


@pytest.mark.parametrize("L,nw,ns,w", [(10, 64, 2000, 5), (16, 256, 400, 8)])
def test_equal_height_matches_oracle(L, nw, ns, w):
    T = 1.4182
    beta, V = 1 / T, L ** 3
    ej, ed, m, lnW, dt = wl.synthetic_series(L=L, T=T, n_walkers=nw, n_samples=ns, seed=3 * L)
    split = int(0.525 * V)
    ref = oracle.equal_height(ed, lnW, 0, beta, split, dt - 0.05, dt + 0.05, n_jack=w)
    got = muca().equal_height(dev(ed), lnW, 0, beta, split, dt - 0.05, dt + 0.05, n_jack=w)
    assert abs(got[0] - ref[0, 0]) <= 1e-9
    assert abs(got[2] - ref[0, 1]) <= 1e-12 * abs(ref[0, 1])
    assert got[4] == tuple(int(v) for v in ref[0, 2:5])
    np.testing.assert_allclose(got[5][:, 0], ref[1:, 0], rtol=0, atol=1e-9)
    np.testing.assert_allclose(got[5][:, 1], ref[1:, 1], rtol=1e-12)
    np.testing.assert_allclose(got[1], jack_err(ref[1:, 0]), rtol=1e-5)
    np.testing.assert_allclose(got[3], jack_err(ref[1:, 1]), rtol=1e-5)


def test_equal_height_full_size_matches_oracle():
    """The reweight workload (4096 walkers x 10^4 samples of L = 32), 10 jackknife blocks."""
    s = wl.REWEIGHT
    ej, ed, m, lnW, dt = wl.synthetic_series()
    beta, V = 1 / s["T"], s["L"] ** 3
    split = int(0.525 * V)
    ref = oracle.equal_height(ed, lnW, 0, beta, split, dt - 0.01, dt + 0.01, n_jack=10)
    got = muca().equal_height(dev(ed), lnW, 0, beta, split, dt - 0.01, dt + 0.01, n_jack=10)
    assert abs(got[0] - ref[0, 0]) <= 1e-9 and abs(got[0] - dt) < 1e-3
    assert abs(got[2] - ref[0, 1]) <= 1e-12 * abs(ref[0, 1])
    np.testing.assert_allclose(got[5][:, 0], ref[1:, 0], rtol=0, atol=1e-9)


def test_equal_height_errors():
    L, T, dt = 10, 1.0, 2.6
    V, beta, lnW, rows, barrier = double_well(L, T, dt)
    with pytest.raises(muca().MucaError) as e:
        muca().equal_height(dev(rows), lnW, 0, beta, int(0.525 * V), dt + 0.01, dt + 0.05)
    assert e.value.code == muca().ERR_INVALID_ARG
    bad = rows.copy()
    bad[2, 5] = V + 3
    with pytest.raises(muca().MucaError) as e:
        muca().equal_height(dev(bad), lnW, 0, beta, int(0.525 * V), dt - 0.05, dt + 0.05)
    assert e.value.code == muca().ERR_WINDOW
