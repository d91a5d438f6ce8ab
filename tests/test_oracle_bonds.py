"""Pins of the oracle's disordered model (reading R16 of the oracle): the
Blume-Capel model with one quenched integer coupling per bond, sampled in the
same multicanonical ensemble in E_Delta.  All run on the CPU.

What fixes it independently of the code:
- unit couplings are the clean model: energies, table and whole runs equal
  the clean oracle's bit for bit;
- couplings 2 at temperature T are the clean model at T / 2 (the same FP64
  acceptance arguments), so runs are identical with E_J doubled;
- energies equal the definition evaluated by the enumeration helper;
- the sampler's stationary law is the exact L = 2 ensemble with the given
  couplings (chi-square over all 3^8 states), and it rejects the clean
  model's law;
- running tallies equal recomputed energies.
"""
import numpy as np
import pytest

import exact
import oracle
from paper_1502_07214_gb300 import workloads as wl

P_MIN = 1e-4


def test_unit_couplings_are_the_clean_model():
    L, T, W, seed = 3, 1.4182, 12, 4
    V = L ** 3
    ones = np.ones((V, 3), dtype=np.int8)
    rng = np.random.default_rng(1)
    for _ in range(5):
        s = rng.integers(-1, 2, V).astype(np.int8)
        np.testing.assert_array_equal(oracle.energies_bonds(L, s, ones), oracle.energies(L, s))
    lnW = rng.normal(0, 1.0, V + 1)
    np.testing.assert_array_equal(oracle.build_table_bonds(L, T, 1, 0, V, lnW),
                                  oracle.build_table(L, T, 0, V, lnW))
    a = oracle.muca_run(L, T, W, seed, 4, 30, n_meas=6, bonds=ones)
    b = oracle.muca_run(L, T, W, seed, 4, 30, n_meas=6)
    for k in ("hist", "lnW", "spins", "tallies", "ts"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)


@pytest.mark.parametrize("recursion", [0, 1])
def test_doubled_couplings_are_the_clean_model_at_half_the_temperature(recursion):
    """exp(-beta (2 dE_J)) at T equals exp(-(2 beta) dE_J) at T / 2, and both
    products are exact in FP64: the runs agree bit for bit, E_J doubled."""
    L, T, W, seed = 4, 2.0, 16, 9
    V = L ** 3
    twos = np.full((V, 3), 2, dtype=np.int8)
    a = oracle.muca_run(L, T, W, seed, 5, 40, n_meas=8, bonds=twos, recursion=recursion)
    b = oracle.muca_run(L, T / 2, W, seed, 5, 40, n_meas=8, recursion=recursion)
    for k in ("hist", "lnW", "spins"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
    np.testing.assert_array_equal(a["tallies"][:, 0], 2 * b["tallies"][:, 0])
    np.testing.assert_array_equal(a["tallies"][:, 1:], b["tallies"][:, 1:])
    np.testing.assert_array_equal(a["ts"][..., 0], 2 * b["ts"][..., 0])


@pytest.mark.parametrize("L", [2, 3])
def test_energies_are_the_definition(L):
    V = L ** 3
    rng = np.random.default_rng(L)
    J = rng.integers(-3, 4, (V, 3)).astype(np.int8)
    st = exact.all_states(L) if L == 2 else rng.integers(-1, 2, (400, V))
    ej, ed, m = exact.state_energies_bonds(st, L, J)
    for k in range(0, len(st), 7 if L == 2 else 1):
        got = oracle.energies_bonds(L, st[k].astype(np.int8), J)
        assert tuple(got) == (ej[k], ed[k], m[k]), k


def independent_final_states(L, T, lnW, J, n_walkers, n_sweeps, seed):
    out = oracle.muca_run(L, T, n_walkers, seed, 0, 0, n_meas=n_sweeps, lnW=lnW, bonds=J,
                          check=True)
    return [(int(a), int(b)) for a, b, _ in out["ts"][:, -1, :]]


@pytest.mark.parametrize("case", ["bimodal", "pm_j", "diluted"])
def test_sampler_exact_enumeration_l2(case):
    """L = 2 under rough weights with three kinds of realisation: bimodal
    couplings 1 and 3, random signs (+-1), and half the bonds cut (0 and 2);
    a chi-square over the joint (E_J, E_Delta) law of all 3^8 states, and the
    clean model's law (what ignoring the couplings would sample) is
    rejected."""
    L, V = 2, 8
    T = {"bimodal": 3.0, "pm_j": 1.2, "diluted": 2.0}[case]
    j1, j2 = {"bimodal": (1, 3), "pm_j": (-1, 1), "diluted": (0, 2)}[case]
    J = wl.random_bonds(L, j1, j2, seed=5)
    assert (J == j1).any() and (J == j2).any()
    lnW = np.random.default_rng(3).normal(0, 1.0, V + 1)
    beta = 1.0 / T
    probs = exact.joint_distribution(L, beta, lnW, J=J)
    keys = independent_final_states(L, T, lnW, J, n_walkers=20000, n_sweeps=24, seed=7)
    _, _, p = exact.chi2_test(keys, probs)
    assert p > P_MIN, p
    # a sampler that ignored the couplings would follow the clean law
    # (exchanging the classes is no test at L = 2 for +-J: the lattice is
    # bipartite, and flipping one sublattice maps J to -J)
    clean = exact.joint_distribution(L, beta, lnW)
    if any(k not in clean for k in keys):
        return  # states the clean model cannot reach: rejected outright
    _, _, pw = exact.chi2_test(keys, clean)
    assert pw < 1e-12, pw


@pytest.mark.parametrize("L", [3, 5])
def test_running_tallies_equal_recomputed(L):
    V = L ** 3
    J = wl.random_bonds(L, 1, 3, seed=L)
    out = oracle.muca_run(L, 3.0, 6, 2, 3, 20, n_meas=10, bonds=J, check=True)
    assert (out["hist"].sum(axis=1) == 6 * 20).all()
    for w in range(6):
        e = oracle.energies_bonds(L, out["spins"][w], J)
        assert tuple(e) == tuple(out["tallies"][w])
    assert np.abs(out["ts"][..., 0]).max() <= 3 * 3 * V


def test_bond_arguments():
    L = 2
    J = np.ones((8, 3), dtype=np.int8)
    J[0, 0] = 9
    with pytest.raises(oracle.OracleError):
        oracle.muca_run(L, 1.0, 2, 1, 1, 1, bonds=J, jmax=8)
    J[0, 0] = 3
    with pytest.raises(oracle.OracleError):  # |J| above the table's jmax
        oracle.muca_run(L, 1.0, 2, 1, 1, 1, bonds=J, jmax=2)
    oracle.muca_run(L, 1.0, 2, 1, 1, 1, bonds=J, jmax=3)
