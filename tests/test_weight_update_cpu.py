"""The library's host-side weight update (muca_weight_update, the function
that the merge and the graph's host node run) against the oracle, bit for
bit, on the CPU: both recursions, histograms with empty bins and runs of
iterations whose accumulated pair weights carry over.  No device work."""
import numpy as np
import pytest

import oracle
from paper_1502_07214_gb300 import muca as m


def histograms(rng, nE, n):
    out = []
    for k in range(n):
        H = rng.integers(0, 3000, nE).astype(np.uint64)
        H[rng.random(nE) < 0.15] = 0
        if k == 0:
            H[nE // 3:nE // 2] = 0  # an unvisited stretch on the first pass
        out.append(H)
    return out


@pytest.mark.parametrize("kind", [m.REC_PLAIN, m.REC_ACCUMULATED])
@pytest.mark.parametrize("nE", [1, 2, 7, 513])
def test_weight_update_equals_oracle(kind, nE):
    rng = np.random.default_rng(nE + 10 * kind)
    lnW_lib = rng.normal(0.0, 2.0, nE)
    lnW_or = lnW_lib.copy()
    acc_lib = np.zeros(max(nE - 1, 1))
    acc_or = acc_lib.copy()
    for H in histograms(rng, nE, 6):
        m.weight_update(kind, H, lnW_lib, acc_lib)
        if kind == m.REC_PLAIN:
            oracle.update_lnW(H, lnW_or)
        else:
            oracle.update_lnW_acc(H, lnW_or, acc_or)
        np.testing.assert_array_equal(lnW_lib, lnW_or)
        np.testing.assert_array_equal(acc_lib, acc_or)


def test_weight_update_errors():
    H = np.ones(5, dtype=np.uint64)
    lnW = np.zeros(5)
    with pytest.raises(m.MucaError) as e:
        m.weight_update(7, H, lnW, np.zeros(4))
    assert e.value.code == m.ERR_INVALID_ARG
    with pytest.raises(m.MucaError) as e:  # the accumulated recursion needs its pair weights
        m.weight_update(m.REC_ACCUMULATED, H, lnW, None)
    assert e.value.code == m.ERR_INVALID_ARG
    with pytest.raises(m.MucaError) as e:
        m.weight_update(m.REC_PLAIN, np.zeros(0, dtype=np.uint64), np.zeros(0))
    assert e.value.code == m.ERR_INVALID_ARG
    m.weight_update(m.REC_PLAIN, H, lnW)  # the plain one does not
    np.testing.assert_array_equal(lnW, np.zeros(5))


@pytest.mark.parametrize("L,T,e_min,e_max", [(2, 1.0, 0, 8), (4, 0.9, 0, 64), (5, 2.0, 30, 90)])
def test_host_table_build_equals_oracle(L, T, e_min, e_max):
    """muca_build_table (host, no context) against the oracle's table on the
    same weights, entry for entry."""
    from paper_1502_07214_gb300 import workloads as wl

    lnW = wl.random_lnW(e_max - e_min + 1, seed=L, scale=2.0, slope=-2.8 / T)
    got = m.build_table(L, T, e_min, e_max, lnW)
    assert np.array_equal(got, oracle.build_table(L, T, e_min, e_max, lnW))


@pytest.mark.parametrize("L,T,jmax,e_min,e_max", [(2, 1.0, 1, 0, 8), (4, 3.0, 3, 10, 60),
                                                  (6, 2.0, 8, 0, 216)])
def test_host_bonds_table_build_equals_oracle(L, T, jmax, e_min, e_max):
    """muca_build_table_bonds (the disordered model's table, host, no
    context) against the oracle's, entry for entry; at jmax = 1 it is the
    clean table."""
    from paper_1502_07214_gb300 import workloads as wl

    lnW = wl.random_lnW(e_max - e_min + 1, seed=L + jmax, scale=2.0, slope=-2.8 / T)
    got = m.build_table_bonds(L, T, jmax, e_min, e_max, lnW)
    assert np.array_equal(got, oracle.build_table_bonds(L, T, jmax, e_min, e_max, lnW))
    if jmax == 1:
        assert np.array_equal(got, m.build_table(L, T, e_min, e_max, lnW))
    with pytest.raises(m.MucaError):
        m.build_table_bonds(L, T, 9, e_min, e_max, lnW)
