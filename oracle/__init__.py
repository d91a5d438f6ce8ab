"""ctypes front-end of the CPU oracle (TEST INFRASTRUCTURE ONLY).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path never does: it shares
no code with the oracle and fails loudly when its own CUDA library is missing.

Every function is a thin numpy wrapper around ``muca_oracle.c``; see that file
for the paper passages and the readings each step follows.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        i32, u32, i64, u64, dbl = (ctypes.c_int32, ctypes.c_uint32, ctypes.c_int64,
                                   ctypes.c_uint64, ctypes.c_double)
        P = ctypes.c_void_p
        L.or_philox4x32_10.argtypes = [P, P, P]
        L.or_philox4x32_10.restype = None
        L.or_init_spins.argtypes = [i32, u32, u32, P]
        L.or_energies.argtypes = [i32, P, P]
        L.or_build_table.argtypes = [i32, dbl, i32, i32, P, P]
        L.or_sweeps.argtypes = [i32, i32, i32, P, u32, u32, u64, i32, P, P, P, P, i32]
        L.or_update_lnW.argtypes = [i32, P, P]
        L.or_update_lnW_acc.argtypes = [i32, P, P, P]
        L.or_muca_run.argtypes = [i32, dbl, i32, i32, i32, u32, u32, i32, i32, i32,
                                  P, P, P, P, P, i32, i32]
        L.or_muca_run_rec.argtypes = [i32, dbl, i32, i32, i32, u32, u32, i32, i32, i32,
                                      P, P, P, P, P, i32, i32, i32, P]
        L.or_muca_run_win.argtypes = [i32, dbl, i32, i32, i32, u32, u32, i32, i32, i32,
                                      P, P, P, P, P, i32, i32, i32, P, i32, i32, dbl, i32, P]
        L.or_energies_bonds.argtypes = [i32, P, P, P]
        L.or_build_table_bonds.argtypes = [i32, dbl, i32, i32, i32, P, P]
        L.or_sweeps_bonds.argtypes = [i32, P, i32, i32, i32, P, u32, u32, u64, i32, P, P, P, P,
                                      i32]
        L.or_muca_run_bonds.argtypes = [i32, dbl, i32, i32, i32, u32, u32, i32, i32, i32,
                                        P, P, P, P, P, i32, i32, i32, P, i32, i32, dbl, i32, P,
                                        P, i32]
        L.or_reweight.argtypes = [P, P, P, i64, P, i32, i32, dbl, i32, P, i32, i32, P]
        L.or_reweight_q.argtypes = [P, P, P, i64, P, i32, i32, dbl, i32, P, i32, i32, P]
        L.or_find_peak.argtypes = [P, P, i64, i32, P, i32, i32, dbl, dbl, dbl, i32, i32, i32, P]
        L.or_equal_height.argtypes = [P, i64, i32, P, i32, i32, dbl, i32, dbl, dbl, i32, i32,
                                      i32, P]
        for f in ("or_init_spins", "or_energies", "or_build_table", "or_sweeps",
                  "or_update_lnW", "or_update_lnW_acc", "or_muca_run", "or_muca_run_rec",
                  "or_muca_run_win", "or_energies_bonds", "or_build_table_bonds",
                  "or_sweeps_bonds", "or_muca_run_bonds",
                  "or_reweight", "or_reweight_q",
                  "or_find_peak", "or_equal_height"):
            getattr(L, f).restype = ctypes.c_int
        _lib = L
    return _lib


class OracleError(RuntimeError):
    pass


def _ck(rc, what):
    if rc != 0:
        raise OracleError(f"{what} failed with code {rc}")


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def init_spins(L, seed, walker_id):
    s = np.zeros(L ** 3, dtype=np.int8)
    _ck(lib().or_init_spins(L, seed, walker_id, _p(s)), "init_spins")
    return s


def energies(L, spins):
    s = np.ascontiguousarray(spins, dtype=np.int8)
    out = np.zeros(3, dtype=np.int64)
    _ck(lib().or_energies(L, _p(s), _p(out)), "energies")
    return out


def build_table(L, T, e_min, e_max, lnW):
    lnW = np.ascontiguousarray(lnW, dtype=np.float64)
    nE = e_max - e_min + 1
    assert lnW.shape == (nE,)
    thr = np.zeros((nE, 3, 25), dtype=np.uint32)
    _ck(lib().or_build_table(L, T, e_min, e_max, _p(lnW), _p(thr)), "build_table")
    return thr


def sweeps(L, e_min, e_max, thr, seed, walker_id, sweep0, n_sweeps, spins, tallies,
           hist=None, record=False, check=False):
    """Run n_sweeps on one walker in place; returns the time series or None."""
    assert spins.dtype == np.int8 and spins.flags.c_contiguous
    assert tallies.dtype == np.int32 and tallies.flags.c_contiguous
    thr = np.ascontiguousarray(thr, dtype=np.uint32)
    ts = np.zeros((n_sweeps, 3), dtype=np.int32) if record else None
    if hist is not None:
        assert hist.dtype == np.uint64 and hist.flags.c_contiguous
    _ck(lib().or_sweeps(L, e_min, e_max, _p(thr), seed, walker_id, sweep0, n_sweeps,
                        _p(spins), _p(tallies), _p(hist), _p(ts), int(check)), "sweeps")
    return ts


def _bonds(L, J, jmax=None):
    J = np.ascontiguousarray(J, dtype=np.int8).reshape(L ** 3, 3)
    if jmax is None:
        jmax = max(1, int(np.abs(J.astype(np.int64)).max()))
    return J, int(jmax)


def energies_bonds(L, spins, J):
    """(E_J, E_Delta, M) of the disordered model (reading R16 of muca_oracle.c);
    J int8 [L^3][3]: couplings of the forward x, y, z bonds of each site."""
    J, _ = _bonds(L, J)
    spins = np.ascontiguousarray(spins, dtype=np.int8)
    out = np.zeros(3, dtype=np.int64)
    _ck(lib().or_energies_bonds(L, _p(spins), _p(J), _p(out)), "energies_bonds")
    return out


def build_table_bonds(L, T, jmax, e_min, e_max, lnW):
    """Table [nE][3][24 jmax + 1] of the disordered model, index dE_J + 12 jmax."""
    lnW = np.ascontiguousarray(lnW, dtype=np.float64)
    nE = e_max - e_min + 1
    assert lnW.shape == (nE,)
    thr = np.zeros((nE, 3, 24 * jmax + 1), dtype=np.uint32)
    _ck(lib().or_build_table_bonds(L, T, jmax, e_min, e_max, _p(lnW), _p(thr)), "build_table_bonds")
    return thr


def sweeps_bonds(L, J, jmax, e_min, e_max, thr, seed, walker_id, sweep0, n_sweeps, spins,
                 tallies, hist=None, record=False, check=False):
    """or_sweeps of the disordered model; spins and tallies updated in place."""
    J, jmax = _bonds(L, J, jmax)
    assert spins.dtype == np.int8 and spins.flags.c_contiguous
    assert tallies.dtype == np.int32 and tallies.flags.c_contiguous
    thr = np.ascontiguousarray(thr, dtype=np.uint32)
    ts = np.zeros((n_sweeps, 3), dtype=np.int32) if record else None
    _ck(lib().or_sweeps_bonds(L, _p(J), jmax, e_min, e_max, _p(thr), seed, walker_id, sweep0,
                              n_sweeps, _p(spins), _p(tallies), _p(hist), _p(ts), int(check)),
        "sweeps_bonds")
    return ts


def update_lnW(H, lnW):
    H = np.ascontiguousarray(H, dtype=np.uint64)
    assert lnW.dtype == np.float64 and lnW.flags.c_contiguous
    _ck(lib().or_update_lnW(len(H), _p(H), _p(lnW)), "update_lnW")


def update_lnW_acc(H, lnW, acc):
    """The accumulated, error-weighted recursion (reading R13 of muca_oracle.c);
    lnW[nE] and the pair weights acc[nE - 1] are updated in place."""
    H = np.ascontiguousarray(H, dtype=np.uint64)
    assert lnW.dtype == np.float64 and lnW.flags.c_contiguous
    assert acc.dtype == np.float64 and acc.flags.c_contiguous and len(acc) == max(len(H) - 1, 1)
    _ck(lib().or_update_lnW_acc(len(H), _p(H), _p(lnW), _p(acc)), "update_lnW_acc")


def flatness(H):
    """Flatness of a merged histogram over its window: (min H / mean H,
    max H / mean H, bins with H > 0); mean = sum / bins; zeros if H is empty."""
    H = np.asarray(H, dtype=np.uint64)
    total = int(H.sum())
    if total == 0:
        return np.zeros(3)
    mean = float(total) / len(H)
    return np.array([float(H.min()) / mean, float(H.max()) / mean, float((H > 0).sum())])


def muca_run(L, T, n_walkers, seed, n_iter, sweeps_per_iter, n_meas=0, e_min=0, e_max=None,
             walker_id0=0, lnW=None, check=False, n_threads=None, want_spins=True, recursion=0,
             acc=None, window=None, grow_flat=0.0, grow_step=0, bonds=None, jmax=None):
    """A whole run of one (L, T) group; returns a dict of numpy arrays.
    recursion 0: lnW -= ln H; 1: the accumulated recursion, whose pair
    weights start from acc (zeros by default) and are returned as "acc".
    window (lo, hi): the walkers' active E_Delta window (reading R15 of
    muca_oracle.c), growing by grow_step bins on each side after an iteration
    whose histogram has min H / mean H >= grow_flat over it; "windows" holds
    the window after every iteration.  Default: [e_min, e_max], fixed.
    bonds int8 [L^3][3]: the disordered model's couplings (reading R16), with
    the table width of jmax (default: the largest |J|); None: the clean model."""
    V = L ** 3
    if e_max is None:
        e_max = V
    nE = e_max - e_min + 1
    lo, hi = (e_min, e_max) if window is None else window
    lnW = np.zeros(nE) if lnW is None else np.array(lnW, dtype=np.float64, copy=True)
    acc = np.zeros(max(nE - 1, 1)) if acc is None else np.array(acc, dtype=np.float64, copy=True)
    hist = np.zeros((max(n_iter, 1), nE), dtype=np.uint64)
    wins = np.zeros((max(n_iter, 1), 2), dtype=np.int32)
    spins = np.zeros((n_walkers, V), dtype=np.int8) if want_spins else None
    tal = np.zeros((n_walkers, 3), dtype=np.int32)
    ts = np.zeros((n_walkers, n_meas, 3), dtype=np.int32) if n_meas > 0 else None
    if n_threads is None:
        n_threads = os.cpu_count() or 1
    J, jm = (None, 0) if bonds is None else _bonds(L, bonds, jmax)
    _ck(lib().or_muca_run_bonds(L, T, n_walkers, e_min, e_max, seed, walker_id0, n_iter,
                                sweeps_per_iter, n_meas, _p(lnW), _p(hist), _p(spins), _p(tal),
                                _p(ts), int(check), n_threads, int(recursion), _p(acc), int(lo),
                                int(hi), float(grow_flat), int(grow_step), _p(wins), _p(J),
                                jm),
        "muca_run")
    return {"lnW": lnW, "hist": hist[:n_iter], "spins": spins, "tallies": tal, "ts": ts,
            "acc": acc, "windows": wins[:n_iter]}


def _rw(fn, e_j, e_d, m, lnW, e_min, beta, V, grid, n_threads):
    e_j = np.ascontiguousarray(e_j, dtype=np.int32).ravel()
    e_d = np.ascontiguousarray(e_d, dtype=np.int32).ravel()
    m = np.ascontiguousarray(m, dtype=np.int32).ravel()
    lnW = np.ascontiguousarray(lnW, dtype=np.float64)
    grid = np.ascontiguousarray(grid, dtype=np.float64)
    out = np.zeros((len(grid), 5))
    if n_threads is None:
        n_threads = os.cpu_count() or 1
    _ck(fn(_p(e_j), _p(e_d), _p(m), len(e_d), _p(lnW), e_min, len(lnW), beta, V, _p(grid),
           len(grid), n_threads, _p(out)), "reweight")
    return out


def reweight(e_j, e_d, m, lnW, e_min, beta, V, grid, n_threads=None):
    """FP64 reweighting; columns <E_J>, <E_Delta>, C, chi, U4."""
    return _rw(lib().or_reweight, e_j, e_d, m, lnW, e_min, beta, V, grid, n_threads)


def reweight_q(e_j, e_d, m, lnW, e_min, beta, V, grid, n_threads=None):
    """binary128 reweighting (rounded to FP64 on output)."""
    return _rw(lib().or_reweight_q, e_j, e_d, m, lnW, e_min, beta, V, grid, n_threads)


def find_peak(e_j, e_d, lnW, e_min, beta, lo, hi, n_iter=60, n_jack=0, n_threads=None):
    """Delta*_L and C*_L by bisection on dC/dDelta (Sec. III) for the full series
    and the n_jack leave-one-block-out subsets.  e_j, e_d are [n_rows][row_len]
    (one row per sweep).  Returns an array [1 + n_jack][2] of (Delta*, C*)."""
    ej = np.ascontiguousarray(e_j, dtype=np.int32)
    ed = np.ascontiguousarray(e_d, dtype=np.int32)
    if ed.ndim == 1:
        ej, ed = ej[None, :], ed[None, :]
    lw = np.ascontiguousarray(lnW, dtype=np.float64)
    out = np.zeros((1 + n_jack, 2))
    nt = n_threads or min(os.cpu_count() or 1, 1 + n_jack)
    _ck(lib().or_find_peak(_p(ej), _p(ed), ed.shape[0], ed.shape[1], _p(lw), e_min, len(lw),
                           beta, lo, hi, n_iter, n_jack, nt, _p(out)), "or_find_peak")
    return out


def equal_height(e_d, lnW, e_min, beta, split, lo, hi, n_iter=60, n_jack=0, n_threads=None):
    """Delta_eqh and the barrier B (equal-height reweighted E_Delta distribution)
    for the full series and the n_jack leave-one-block-out subsets.  e_d is
    [n_rows][row_len].  Returns [1 + n_jack][5]: Delta_eqh, B, E of the left
    peak, E of the right peak, E of the minimum between them."""
    ed = np.ascontiguousarray(e_d, dtype=np.int32)
    if ed.ndim == 1:
        ed = ed[None, :]
    lw = np.ascontiguousarray(lnW, dtype=np.float64)
    out = np.zeros((1 + n_jack, 5))
    nt = n_threads or min(os.cpu_count() or 1, 1 + n_jack)
    _ck(lib().or_equal_height(_p(ed), ed.shape[0], ed.shape[1], _p(lw), e_min, len(lw), beta,
                              split, lo, hi, n_iter, n_jack, nt, _p(out)), "or_equal_height")
    return out
