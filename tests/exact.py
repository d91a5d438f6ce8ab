"""Brute-force enumeration of small Blume-Capel lattices (test helper).

Written directly from the model's definition (Eq. 1): spins in {-1, 0, +1} on an
L^3 periodic simple-cubic lattice, E_J = -sum over nearest-neighbour bonds,
E_Delta = sum s_i^2, M = sum s_i.  Bonds are the three forward bonds of each
site (at L = 2 both bonds of a pair count, as the six-neighbour local field
does).  Nothing here is shared with the oracle or with the CUDA library.
"""
import itertools

import numpy as np


def forward_neighbours(L):
    nb = np.zeros((L ** 3, 3), dtype=np.int64)
    for z, y, x in itertools.product(range(L), repeat=3):
        i = x + L * (y + L * z)
        nb[i, 0] = (x + 1) % L + L * (y + L * z)
        nb[i, 1] = x + L * ((y + 1) % L + L * z)
        nb[i, 2] = x + L * (y + L * ((z + 1) % L))
    return nb


def all_states(L, values=(-1, 0, 1)):
    V = L ** 3
    k = len(values)
    idx = np.arange(k ** V, dtype=np.int64)
    st = np.zeros((k ** V, V), dtype=np.int64)
    vals = np.asarray(values, dtype=np.int64)
    for i in range(V):
        st[:, i] = vals[idx % k]
        idx //= k
    return st


def state_energies(st, L):
    nb = forward_neighbours(L)
    ej = np.zeros(len(st), dtype=np.int64)
    for mu in range(3):
        ej -= (st * st[:, nb[:, mu]]).sum(axis=1)
    ed = (st * st).sum(axis=1)
    m = st.sum(axis=1)
    return ej, ed, m


def state_energies_bonds(st, L, J):
    """(E_J, E_Delta, M) with a coupling per bond: E_J = -sum over the forward
    bonds (i, mu) of J[i, mu] s_i s_{i+mu}."""
    nb = forward_neighbours(L)
    J = np.asarray(J, dtype=np.int64).reshape(L ** 3, 3)
    ej = np.zeros(len(st), dtype=np.int64)
    for mu in range(3):
        ej -= (J[:, mu] * st * st[:, nb[:, mu]]).sum(axis=1)
    ed = (st * st).sum(axis=1)
    m = st.sum(axis=1)
    return ej, ed, m


def joint_distribution(L, beta, lnW, e_min=0, values=(-1, 0, 1), J=None):
    """Exact P(E_J, E_Delta) of the ensemble exp(-beta E_J) W(E_Delta), with
    one coupling per bond if J [L^3][3] is given (else J = 1).

    Returns a dict {(E_J, E_Delta): probability}."""
    st = all_states(L, values)
    ej, ed, _ = state_energies(st, L) if J is None else state_energies_bonds(st, L, J)
    logw = -beta * ej + np.asarray(lnW)[ed - e_min]
    w = np.exp(logw - logw.max())
    w /= w.sum()
    out = {}
    for a, b, p in zip(ej, ed, w):
        out[(int(a), int(b))] = out.get((int(a), int(b)), 0.0) + float(p)
    return out


def canonical_averages(L, beta, delta):
    """Exact canonical <E_J>, <E_Delta>, C, chi, U4 at (beta, Delta) (Eq. 2, Eq. 6)."""
    st = all_states(L)
    ej, ed, m = state_energies(st, L)
    V = L ** 3
    logw = -beta * (ej + delta * ed)
    w = np.exp(logw - logw.max())
    w /= w.sum()
    mj = (w * ej).sum()
    md = (w * ed).sum()
    mjd = (w * ej * ed).sum()
    mm = m / V
    m1 = (w * np.abs(mm)).sum()
    m2 = (w * mm ** 2).sum()
    m4 = (w * mm ** 4).sum()
    return np.array([mj, md, -beta * (mjd - mj * md), beta * V * (m2 - m1 * m1),
                     1 - m4 / (3 * m2 * m2)])


def chi2_test(samples_keys, probs, min_expected=5.0):
    """Pearson chi-square of observed keys against exact probabilities.

    Cells with small expectation are pooled.  Returns (chi2, dof, p_value)."""
    from scipy import stats

    n = len(samples_keys)
    counts = {}
    for k in samples_keys:
        counts[k] = counts.get(k, 0) + 1
    for k in counts:
        assert k in probs and probs[k] > 0, f"sampled impossible cell {k}"
    keys = sorted(probs, key=lambda k: probs[k])
    obs, exp = [], []
    po, pe = 0.0, 0.0
    for k in keys:
        e = probs[k] * n
        o = counts.get(k, 0)
        if e < min_expected:
            po += o
            pe += e
            if pe >= min_expected:
                obs.append(po)
                exp.append(pe)
                po, pe = 0.0, 0.0
        else:
            obs.append(o)
            exp.append(e)
    if pe > 0:
        obs[-1] += po
        exp[-1] += pe
    obs = np.array(obs, dtype=float)
    exp = np.array(exp, dtype=float)
    chi2 = float(((obs - exp) ** 2 / exp).sum())
    dof = len(obs) - 1
    return chi2, dof, float(stats.chi2.sf(chi2, dof))
