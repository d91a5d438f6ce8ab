"""muca_reweight_noalloc, the reweighting entry point that allocates no device
memory (for callers that cannot allocate at the point of the call, such as a
service under a fixed device-memory budget or a binding without a device
allocator), against muca_reweight on the same inputs, twice in a row (the
fixed working array is shared between calls and must be cleared by each), and
against the FP64 oracle directly.  This file is collected last so that a run
stopping at the first failure has run everything else."""
import numpy as np
import pytest

import oracle
from paper_1502_07214_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

TOL = {64: 1e-12, 32: 1e-5}


def muca():
    from paper_1502_07214_gb300 import muca as m

    return m


def rel_err(got, ref):
    scale = np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max(axis=0, keepdims=True))
    scale = np.where(scale == 0, 1.0, scale)
    return np.abs(got - ref) / scale


@pytest.mark.parametrize("precision", [64, 32])
def test_noalloc_matches_reweight_twice(precision):
    L, T = 16, 1.4182
    ej, ed, m, lnW, dt = wl.synthetic_series(L=L, T=T, n_walkers=128, n_samples=200, seed=17)
    dev = [torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32).ravel()).cuda()
           for a in (ej, ed, m)]
    grid = wl.delta_grid(dt, 0.05, 257)
    ref = muca().reweight(*dev, lnW, 0, 1 / T, L ** 3, grid, precision)
    first = muca().reweight(*dev, lnW, 0, 1 / T, L ** 3, grid, precision, no_alloc=True)
    second = muca().reweight(*dev, lnW, 0, 1 / T, L ** 3, grid, precision, no_alloc=True)
    assert (rel_err(first, ref) <= TOL[precision]).all()
    assert (rel_err(second, ref) <= TOL[precision]).all()


def test_noalloc_after_a_different_problem():
    """A smaller problem after a larger one: the left-over contents of the
    shared array must not leak into the result."""
    big = wl.synthetic_series(L=32, T=1.0, n_walkers=64, n_samples=100, seed=3)
    small = wl.synthetic_series(L=8, T=2.0, n_walkers=64, n_samples=300, seed=4)
    for (ej, ed, m, lnW, dt), L, T in ((big, 32, 1.0), (small, 8, 2.0)):
        dev = [torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32).ravel()).cuda()
               for a in (ej, ed, m)]
        grid = wl.delta_grid(dt, 0.05, 64)
        ref = muca().reweight(*dev, lnW, 0, 1 / T, L ** 3, grid, 64)
        got = muca().reweight(*dev, lnW, 0, 1 / T, L ** 3, grid, 64, no_alloc=True)
        assert (rel_err(got, ref) <= TOL[64]).all()


def test_noalloc_rejects_problems_beyond_its_array():
    V = 48 ** 3
    ed = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(muca().MucaError) as e:
        muca().reweight(ed, ed, ed, np.zeros(V + 1), 0, 1.0, V, np.linspace(2, 3, 16), 64,
                        no_alloc=True)
    assert e.value.code == muca().ERR_INVALID_ARG


@pytest.mark.parametrize("precision", [64, 32])
def test_noalloc_matches_the_oracle(precision):
    """The same series reweighted by the FP64 oracle on the host: FP64 within
    1e-12 and FP32 within 1e-5 per observable and Delta point."""
    L, T = 12, 1.0
    ej, ed, m, lnW, dt = wl.synthetic_series(L=L, T=T, n_walkers=96, n_samples=150, seed=23)
    dev = [torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32).ravel()).cuda()
           for a in (ej, ed, m)]
    grid = wl.delta_grid(dt, 0.05, 129)
    want = oracle.reweight(ej, ed, m, lnW, 0, 1 / T, L ** 3, grid)
    got = muca().reweight(*dev, lnW, 0, 1 / T, L ** 3, grid, precision, no_alloc=True)
    assert (rel_err(got, want) <= TOL[precision]).all()


def test_noalloc_allocates_no_device_memory():
    """After a first call (which may load the library's device code and its
    fixed array), further calls leave the device's free memory unchanged."""
    L, T = 16, 1.4182
    ej, ed, m, lnW, dt = wl.synthetic_series(L=L, T=T, n_walkers=128, n_samples=100, seed=5)
    dev = [torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32).ravel()).cuda()
           for a in (ej, ed, m)]
    grid = wl.delta_grid(dt, 0.05, 200)
    for p in (64, 32):
        muca().reweight(*dev, lnW, 0, 1 / T, L ** 3, grid, p, no_alloc=True)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for p in (64, 32, 64):
        muca().reweight(*dev, lnW, 0, 1 / T, L ** 3, grid, p, no_alloc=True)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
