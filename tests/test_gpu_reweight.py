"""GPU reweighting (Eq. 3, Eq. 6) against the CPU oracle.

Tolerances (per observable, every Delta_k): FP64 within 1e-12 and FP32
within 1e-5, as relative errors against the FP64 oracle with the denominator
max(|ref_k|, 1e-3 max_k |ref_k|) so that an observable crossing zero (C far
from the transition) is judged on the scale of its own curve.
"""
import numpy as np
import pytest

import oracle
from paper_1502_07214_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

TOL = {64: 1e-12, 32: 1e-5}
NAMES = ["E_J", "E_Delta", "C", "chi", "U4"]


def muca():
    from paper_1502_07214_gb300 import muca as m

    return m


def rel_err(got, ref):
    scale = np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max(axis=0, keepdims=True))
    scale = np.where(scale == 0, 1.0, scale)
    return np.abs(got - ref) / scale


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32).ravel()).cuda()


def series(L, n_walkers, n_samples, seed, T=1.4182):
    ej, ed, m, lnW, dt = wl.synthetic_series(L=L, T=T, n_walkers=n_walkers, n_samples=n_samples,
                                             seed=seed)
    return ej, ed, m, lnW, dt


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("L,nw,ns", [(8, 256, 400), (12, 333, 101), (16, 64, 1000)])
def test_reweight_matches_oracle(precision, L, nw, ns):
    T = 1.4182
    beta = 1 / T
    ej, ed, m, lnW, dt = series(L, nw, ns, seed=L)
    grid = wl.delta_grid(dt, 0.05, 97)
    ref = oracle.reweight(ej, ed, m, lnW, 0, beta, L ** 3, grid)
    got = muca().reweight(dev(ej), dev(ed), dev(m), lnW, 0, beta, L ** 3, grid, precision)
    err = rel_err(got, ref)
    worst = dict(zip(NAMES, err.max(axis=0)))
    assert (err <= TOL[precision]).all(), worst


def test_against_binary128():
    """Both precisions against the literal definition in binary128; FP64 within
    the FP64 oracle's own bound (1e-10, see the oracle pins), FP32 within 1e-5."""
    L, T = 10, 1.4182
    ej, ed, m, lnW, dt = series(L, 128, 300, seed=3)
    grid = wl.delta_grid(dt, 0.05, 33)
    q = oracle.reweight_q(ej, ed, m, lnW, 0, 1 / T, L ** 3, grid)
    got = muca().reweight(dev(ej), dev(ed), dev(m), lnW, 0, 1 / T, L ** 3, grid, 64)
    assert (rel_err(got, q) <= 1e-10).all()
    got = muca().reweight(dev(ej), dev(ed), dev(m), lnW, 0, 1 / T, L ** 3, grid, 32)
    assert (rel_err(got, q) <= 1e-5).all()


def test_strided_layout_of_the_context_series():
    """[sample][field][walker] rows with a stride, as the context records them."""
    L, T, W, S = 6, 1.0, 45, 70
    ej, ed, m, lnW, dt = series(L, W, S, seed=9, T=T)
    packed = np.stack([ej, ed, m], axis=1).astype(np.int32)  # [S][3][W]
    buf = torch.from_numpy(packed.ravel()).cuda()
    base = buf.data_ptr()
    grid = wl.delta_grid(dt, 0.05, 16)
    got = muca().reweight(base, base + 4 * W, base + 8 * W, lnW, 0, 1 / T, L ** 3, grid, 64,
                          n_rows=S, row_len=W, row_stride=3 * W)
    ref = oracle.reweight(ej, ed, m, lnW, 0, 1 / T, L ** 3, grid)
    assert (rel_err(got, ref) <= 1e-12).all()


def test_context_series_end_to_end():
    """A recorded run reweighted on the GPU equals the oracle's reweighting of
    the oracle's own run (the two series are bit-identical)."""
    L, T, W, seed = 4, 1.4182, 64, 13
    c = muca().Context([{"L": L, "T": T, "n_walkers": W}], seed=seed)
    for _ in range(4):
        c.sweep_iter(50)
        c.merge_update()
    c.reserve_timeseries(200)
    c.sweep_iter(200, record=True)
    grid = np.linspace(2.0, 3.5, 40)
    got64 = muca().reweight_context(c, 0, grid, 64)
    got32 = muca().reweight_context(c, 0, grid, 32)
    c.close()
    ref = oracle.muca_run(L, T, W, seed, 4, 50, n_meas=200)
    ts = ref["ts"]
    want = oracle.reweight(ts[..., 0], ts[..., 1], ts[..., 2], ref["lnW"], 0, 1 / T, L ** 3, grid)
    assert (rel_err(got64, want) <= 1e-12).all()
    assert (rel_err(got32, want) <= 1e-5).all()


def test_degenerate_inputs():
    # one sample; all samples in one E_Delta bin (C = 0, chi from |m| only)
    V, beta = 64, 0.5
    lnW = np.zeros(V + 1)
    got = muca().reweight(dev([-10]), dev([20]), dev([-4]), lnW, 0, beta, V, [1.0, 2.0], 64)
    assert np.allclose(got[:, 0], -10) and np.allclose(got[:, 1], 20)
    assert np.allclose(got[:, 2], 0) and np.allclose(got[:, 3], 0)
    ed = np.full(500, 33)
    ej = np.arange(500) - 250
    m = (np.arange(500) % 7) - 3
    for p in (64, 32):
        got = muca().reweight(dev(ej), dev(ed), dev(m), lnW, 0, beta, V, [0.5, 3.0], p)
        ref = oracle.reweight(ej, ed, m, lnW, 0, beta, V, [0.5, 3.0])
        assert np.allclose(got[:, 2], 0, atol=1e-9)
        assert np.allclose(got[:, [0, 1, 3, 4]], ref[:, [0, 1, 3, 4]], rtol=TOL[p], atol=1e-12)
    # an E_Delta outside [e_min, e_min + n_e) is an error, not a fault
    with pytest.raises(muca().MucaError) as e:
        muca().reweight(dev([0, 1]), dev([5, 70]), dev([0, 0]), lnW, 0, beta, V, [1.0], 64)
    assert e.value.code == muca().ERR_WINDOW
    with pytest.raises(muca().MucaError):
        muca().reweight(dev([0]), dev([5]), dev([0]), lnW, 0, beta, V, [1.0], 16)


def test_full_size_reweight_sampled_grid_points():
    """4096 walkers x 10^4 samples of an L=32 series, 4096 grid points: the
    oracle recomputes a sample of grid points."""
    s = wl.REWEIGHT
    ej, ed, m, lnW, dt = wl.synthetic_series()
    beta = 1 / s["T"]
    V = s["L"] ** 3
    grid = wl.delta_grid(dt)
    e_j, e_d, mm = dev(ej), dev(ed), dev(m)
    got64 = muca().reweight(e_j, e_d, mm, lnW, 0, beta, V, grid, 64)
    got32 = muca().reweight(e_j, e_d, mm, lnW, 0, beta, V, grid, 32)
    ks = np.array([0, 1, 1500, 2047, 2048, 3333, 4095])
    ref = oracle.reweight(ej, ed, m, lnW, 0, beta, V, grid[ks])
    full_scale = np.abs(got64).max(axis=0, keepdims=True)
    for got, p in ((got64, 64), (got32, 32)):
        sc = np.maximum(np.abs(ref), 1e-3 * full_scale)
        err = np.abs(got[ks] - ref) / sc
        assert (err <= TOL[p]).all(), (p, dict(zip(NAMES, err.max(axis=0))))
    assert np.isfinite(got64).all() and np.isfinite(got32).all()


def test_bucketed_sums_equal_direct_sums():
    """``muca_reweight`` forms the per-bin integer sums through buckets of bins
    (records summed in shared memory); ``muca_reweight_noalloc`` adds every
    sample to the global sums.  Both sums are exact, so the results must be
    bit-identical: here with samples whose E_J or |M| are too large for a
    record, and with more samples (2^26 + 65536) than one bucketed pass takes."""
    V, n_e = 4999, 5000
    n_rows, row_len = 16400, 4096
    n = n_rows * row_len
    g = torch.Generator(device="cuda").manual_seed(11)
    e_d = torch.randint(0, n_e, (n,), device="cuda", dtype=torch.int32, generator=g)
    e_j = torch.randint(-3 * V, 3 * V + 1, (n,), device="cuda", dtype=torch.int32, generator=g)
    m = torch.randint(-V, V + 1, (n,), device="cuda", dtype=torch.int32, generator=g)
    big = torch.randint(0, n, (4096,), device="cuda", generator=g)
    e_j[big[:2048]] = torch.randint(1 << 20, 1 << 26, (2048,), device="cuda", dtype=torch.int32,
                                    generator=g)
    m[big[2048:]] = -torch.randint((1 << 18) + 1, 1 << 22, (2048,), device="cuda",
                                   dtype=torch.int32, generator=g)
    lnW = wl.random_lnW(n_e, seed=4, scale=3.0, slope=-0.4)
    grid = np.linspace(0.2, 0.6, 13)
    for p in (64, 32):
        a = muca().reweight(e_j, e_d, m, lnW, 0, 0.7, V, grid, p, n_rows=n_rows,
                            row_len=row_len, row_stride=row_len)
        b = muca().reweight(e_j, e_d, m, lnW, 0, 0.7, V, grid, p, n_rows=n_rows,
                            row_len=row_len, row_stride=row_len, no_alloc=True)
        assert np.isfinite(a).all()
        assert np.array_equal(a, b), p


def _context_layout(ej, ed, m):
    """[sample][field][walker] rows (row stride 3 x walkers), as a context records them."""
    packed = np.stack([ej, ed, m], axis=1).astype(np.int32)
    return torch.from_numpy(packed.ravel()).cuda()


def test_bucketed_sums_ragged_rows_and_wide_windows():
    """Stage A's bucketed path against the direct sums and the oracle on the
    shapes its partition has to get right: rows that are not a whole number
    of 4096-sample chunks in the context's strided layout, every bucket of a
    32769-bin window (bit-identical to ``muca_reweight_noalloc``), a 262145-bin
    window (L = 64: 257 buckets, some empty) and one of more than 1024 buckets
    (summed directly) against the FP64 oracle, and all samples in one bin."""
    rng = np.random.default_rng(21)
    beta = 0.7
    # 32769 bins, rows of 5000 walkers (one full chunk and a ragged one)
    S, W, n_e = 700, 5000, 32769
    ed = rng.integers(0, n_e, (S, W))
    ej = rng.integers(-3 * (n_e - 1), 3 * (n_e - 1) + 1, (S, W))
    m = rng.integers(-(n_e - 1), n_e, (S, W))
    buf = _context_layout(ej, ed, m)
    base = buf.data_ptr()
    lnW = wl.random_lnW(n_e, seed=5, scale=2.0, slope=-0.3)
    grid = np.linspace(0.2, 0.6, 9)
    for p in (64, 32):
        kw = dict(n_rows=S, row_len=W, row_stride=3 * W)
        a = muca().reweight(base, base + 4 * W, base + 8 * W, lnW, 0, beta, n_e - 1, grid, p, **kw)
        b = muca().reweight(base, base + 4 * W, base + 8 * W, lnW, 0, beta, n_e - 1, grid, p,
                            no_alloc=True, **kw)
        assert np.isfinite(a).all() and np.array_equal(a, b), p
    # 262145 bins, samples only in the lower 3/5 of the window (empty buckets above)
    S, W, n_e = 300, 4100, 64 ** 3 + 1
    ed = rng.integers(0, (3 * n_e) // 5, (S, W))
    ej = rng.integers(-3 * (n_e - 1), 3 * (n_e - 1) + 1, (S, W))
    m = np.clip(rng.integers(-(n_e - 1), n_e, (S, W)), -ed, ed)
    buf = _context_layout(ej, ed, m)
    base = buf.data_ptr()
    lnW = wl.random_lnW(n_e, seed=6, scale=1.0, slope=-0.35)
    grid = np.linspace(0.3, 0.45, 5)
    ref = oracle.reweight(ej, ed, m, lnW, 0, beta, n_e - 1, grid)
    for p in (64, 32):
        got = muca().reweight(base, base + 4 * W, base + 8 * W, lnW, 0, beta, n_e - 1, grid, p,
                              n_rows=S, row_len=W, row_stride=3 * W)
        assert (rel_err(got, ref) <= TOL[p]).all(), (p, rel_err(got, ref).max(axis=0))
    # a window of 1026 buckets: the direct path
    n_e, S, W = (1 << 21) + 2049, 64, 1000
    ed = rng.integers(0, n_e, (S, W))
    ej = rng.integers(-1000, 1001, (S, W))
    m = rng.integers(-1000, 1001, (S, W))
    lnW = wl.random_lnW(n_e, seed=7, scale=0.01, slope=-0.002)
    grid = np.linspace(0.001, 0.003, 3)
    ref = oracle.reweight(ej, ed, m, lnW, 0, beta, n_e - 1, grid)
    got = muca().reweight(dev(ej), dev(ed), dev(m), lnW, 0, beta, n_e - 1, grid, 64)
    assert (rel_err(got, ref) <= TOL[64]).all(), rel_err(got, ref).max(axis=0)
    # 3 x 10^6 samples in one bin (one thread sums a whole tile)
    n = 3_000_000
    ed = np.full(n, 33)
    ej = rng.integers(-300, 301, n)
    m = rng.integers(-64, 65, n)
    lnW = np.zeros(65)
    a = muca().reweight(dev(ej), dev(ed), dev(m), lnW, 0, 0.5, 64, [0.5, 3.0], 64)
    b = muca().reweight(dev(ej), dev(ed), dev(m), lnW, 0, 0.5, 64, [0.5, 3.0], 64, no_alloc=True)
    assert np.array_equal(a, b)
    assert np.allclose(a[:, 0], ej.mean(), rtol=1e-12)
