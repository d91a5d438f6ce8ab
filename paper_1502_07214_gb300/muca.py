"""Thin Python binding of ``libmuca.so`` (the C ABI in ``include/muca.h``).

Argument marshalling only: every step of the simulation and of the
reweighting runs in the library's CUDA kernels.  Device buffers handed to the
library are torch CUDA tensors (``data_ptr()``), streams are torch streams
(``cuda_stream``).  There is no CPU fallback: if the library cannot be loaded
the calls raise.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmuca.so")

OK = 0
ERR_INVALID_ARG = -1
ERR_CUDA = -2
ERR_OOM = -3
ERR_TIMEOUT = -4
ERR_TALLY_MISMATCH = -5
ERR_NOT_SUPPORTED = -6
ERR_WINDOW = -7
ERR_IO = -8

RES_AUTO, RES_GLOBAL, RES_SMEM, RES_SPLIT, RES_SCAN, RES_BONDS = 0, 1, 2, 3, 4, 5
REC_PLAIN, REC_ACCUMULATED = 0, 1
DEBUG_TALLY_CHECK = 1
NK = 25
MAX_L = 64  # largest linear size (MUCA_MAX_L)
MAX_JMAX = 8  # largest |coupling| of the disordered model (MUCA_MAX_JMAX)


class MucaError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class Group(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("T", ctypes.c_double), ("n_walkers", ctypes.c_int32),
                ("e_min", ctypes.c_int32), ("e_max", ctypes.c_int32)]


class Options(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint32), ("debug_flags", ctypes.c_int32),
                ("residency", ctypes.c_int32), ("walkers_per_block", ctypes.c_int32),
                ("lanes_per_walker", ctypes.c_int32), ("shard_rank", ctypes.c_int32),
                ("shard_count", ctypes.c_int32)]


_lib = None

# exported symbols and their argument types
_P = ctypes.c_void_p
_I32, _I64, _U64, _D = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
SIGNATURES = {
    "muca_init": [_P, ctypes.c_int, _P, _P, _P],
    "muca_destroy": [_P],
    "muca_last_error": [_P],
    "muca_sync": [_P],
    "muca_sweep_iter": [_P, ctypes.c_int, ctypes.c_int],
    "muca_merge_update": [_P],
    "muca_run_graph": [_P, ctypes.c_int, ctypes.c_int],
    "muca_weight_update": [_I32, _I32, _P, _P, _P],
    "muca_set_recursion": [_P, _I32],
    "muca_get_flatness": [_P, ctypes.c_int, _P],
    "muca_iterate": [_P, _I32, _I32, _D, _P],
    "muca_set_window": [_P, ctypes.c_int, _I32, _I32, _D, _I32],
    "muca_set_bonds": [_P, ctypes.c_int, _P, _I32],
    "muca_build_table_bonds": [_I32, _D, _I32, _I32, _I32, _P, _P],
    "muca_probe_int": [_I32, _I32, _P, _P, _P],
    "muca_probe_l2_read": [_I64, _I32, _P, _P, _P],
    "muca_get_window": [_P, ctypes.c_int, _P],
    "muca_reweight": [_P, _P, _P, _I64, _I32, _I64, _P, _I32, _I32, _D, _I32, _P, _I32, _I32,
                      _P, _P],
    "muca_reweight_noalloc": [_P, _P, _P, _I64, _I32, _I64, _P, _I32, _I32, _D, _I32, _P, _I32,
                              _I32, _P, _P],
    "muca_find_peak": [_P, _P, _I64, _I32, _I64, _P, _I32, _I32, _D, _D, _D, _I32, _I32, _P, _P],
    "muca_equal_height": [_P, _I64, _I32, _I64, _P, _I32, _I32, _D, _I32, _D, _D, _I32, _I32, _P,
                          _P],
    "muca_reserve_timeseries": [_P, _I64],
    "muca_timeseries_device": [_P, ctypes.c_int, _P, _P],
    "muca_get_timeseries": [_P, ctypes.c_int, _P],
    "muca_get_sweep_count": [_P, ctypes.c_int, _P],
    "muca_get_lnW": [_P, ctypes.c_int, _P],
    "muca_set_lnW": [_P, ctypes.c_int, _P],
    "muca_get_table": [_P, ctypes.c_int, _P],
    "muca_set_table": [_P, ctypes.c_int, _P],
    "muca_get_hist": [_P, ctypes.c_int, _P],
    "muca_set_hist": [_P, ctypes.c_int, _P],
    "muca_get_hist_device": [_P, ctypes.c_int, _P],
    "muca_set_hist_device": [_P, ctypes.c_int, _P],
    "muca_get_walkers": [_P, ctypes.c_int, _P, _P],
    "muca_build_table": [_I32, _D, _I32, _I32, _P, _P],
    "muca_get_state": [_P, ctypes.c_int, _P, _P],
    "muca_set_state": [_P, ctypes.c_int, _P],
    "muca_check_tallies": [_P],
    "muca_get_config": [_P, ctypes.c_int, _P, _P, _P],
    "muca_checkpoint": [_P, ctypes.c_char_p],
    "muca_restore": [_P, ctypes.c_char_p],
}


def lib(path=None):
    """Load libmuca.so (building it first if it is missing); raises on failure."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        from . import build as _build
        _build.build()
    L = ctypes.CDLL(path)
    for name, argt in SIGNATURES.items():
        f = getattr(L, name)
        f.argtypes = argt
        f.restype = ctypes.c_int
    L.muca_destroy.restype = None
    L.muca_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def last_error(ctx=None):
    return lib().muca_last_error(ctx).decode()


def _ck(rc, ctx=None):
    if rc != OK:
        raise MucaError(rc, last_error(ctx))


def _np_ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _stream_ptr(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream))


def build_table_bonds(L, T, jmax, e_min, e_max, lnW):
    """The disordered model's table [n_e][3][24 jmax + 1] on the host."""
    lnW = np.ascontiguousarray(lnW, dtype=np.float64)
    out = np.zeros((e_max - e_min + 1, 3, 24 * jmax + 1), dtype=np.uint32)
    _ck(lib().muca_build_table_bonds(int(L), float(T), int(jmax), int(e_min), int(e_max),
                                     _np_ptr(lnW), _np_ptr(out)))
    return out


def probe_int(kind, iters=2048, stream=None):
    """Integer instruction rate of one probe kind (``muca_probe_int``):
    (updates per second, best launch in ms)."""
    ops, ms = ctypes.c_double(), ctypes.c_double()
    rc = lib().muca_probe_int(int(kind), int(iters), ctypes.byref(ops), ctypes.byref(ms),
                              _stream_ptr(stream))
    if rc != 0:
        raise MucaError(ERR_CUDA if rc == -2 else ERR_INVALID_ARG, f"muca_probe_int: {rc}")
    return ops.value, ms.value


def probe_l2_read(n_bytes=32 << 20, reps=64, stream=None):
    """L2 read bandwidth over a buffer of n_bytes (``muca_probe_l2_read``):
    (bytes per second, best launch in ms)."""
    bw, ms = ctypes.c_double(), ctypes.c_double()
    rc = lib().muca_probe_l2_read(int(n_bytes), int(reps), ctypes.byref(bw), ctypes.byref(ms),
                                  _stream_ptr(stream))
    if rc != 0:
        raise MucaError(ERR_CUDA if rc == -2 else ERR_INVALID_ARG, f"muca_probe_l2_read: {rc}")
    return bw.value, ms.value


def build_table(L, T, e_min, e_max, lnW):
    """The acceptance-threshold table of a weight function, built on the host
    (``muca_build_table``): uint32 [n_e][3][NK]."""
    lnW = np.ascontiguousarray(lnW, dtype=np.float64)
    n_e = e_max - e_min + 1
    assert lnW.shape == (n_e,)
    out = np.zeros((n_e, 3, NK), dtype=np.uint32)
    _ck(lib().muca_build_table(int(L), float(T), int(e_min), int(e_max), _np_ptr(lnW),
                               _np_ptr(out)))
    return out


def weight_update(kind, hist, lnW, acc=None):
    """One host-side weight update (muca_weight_update): lnW (float64) and,
    for REC_ACCUMULATED, the pair weights acc (float64, len(hist) - 1) are
    updated in place."""
    hist = np.ascontiguousarray(hist, dtype=np.uint64)
    assert lnW.dtype == np.float64 and lnW.flags.c_contiguous and len(lnW) == len(hist)
    if acc is not None:
        assert acc.dtype == np.float64 and acc.flags.c_contiguous
        assert len(acc) >= len(hist) - 1
    _ck(lib().muca_weight_update(int(kind), len(hist), _np_ptr(hist), _np_ptr(lnW),
                                 None if acc is None else _np_ptr(acc)))


class Context:
    """A set of (L, T) walker groups on one GPU (``muca_init`` .. ``muca_destroy``)."""

    def __init__(self, groups, seed=0, debug_flags=0, residency=RES_AUTO, walkers_per_block=0,
                 lanes_per_walker=0, stream=None, shard=(0, 0)):
        """groups: dicts with L, T, n_walkers (and optionally e_min, e_max);
        shard = (rank, count): with count > 1 the context holds shard `rank`
        of every group's n_walkers walkers (the ``n_walkers`` of ``specs`` is
        then the shard's own count)."""
        L = lib()
        self.specs = []
        arr = (Group * len(groups))()
        for i, g in enumerate(groups):
            g = dict(g)
            e_max = g.get("e_max", -1)
            arr[i] = Group(int(g["L"]), float(g["T"]), int(g["n_walkers"]), int(g.get("e_min", 0)),
                           int(e_max))
            V = int(g["L"]) ** 3
            self.specs.append({"L": int(g["L"]), "T": float(g["T"]), "n_walkers": int(g["n_walkers"]),
                               "e_min": int(g.get("e_min", 0)),
                               "e_max": V if e_max < 0 else int(e_max), "V": V})
        opt = Options(seed, debug_flags, residency, walkers_per_block, lanes_per_walker,
                      int(shard[0]), int(shard[1]))
        self._stream = _stream_ptr(stream)
        self._ctx = ctypes.c_void_p()
        _ck(L.muca_init(ctypes.cast(arr, _P), len(groups), ctypes.byref(opt), self._stream,
                        ctypes.byref(self._ctx)))
        for g, sp in enumerate(self.specs):
            n = ctypes.c_int32()
            w0 = ctypes.c_uint32()
            self._c(L.muca_get_walkers(self._ctx, g, ctypes.byref(n), ctypes.byref(w0)))
            sp["n_walkers_total"] = sp["n_walkers"]
            sp["n_walkers"] = n.value
            sp["first_walker"] = w0.value

    # -- lifetime
    def close(self):
        if self._ctx:
            lib().muca_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _c(self, rc):
        _ck(rc, self._ctx)

    def n_e(self, g):
        if not 0 <= g < len(self.specs):
            raise MucaError(ERR_INVALID_ARG, f"group {g} out of range [0, {len(self.specs)})")
        s = self.specs[g]
        return s["e_max"] - s["e_min"] + 1

    # -- hot path
    def sweep_iter(self, n_sweeps, record=False):
        self._c(lib().muca_sweep_iter(self._ctx, n_sweeps, int(bool(record))))

    def merge_update(self):
        self._c(lib().muca_merge_update(self._ctx))

    def run_graph(self, n_iters, sweeps_per_iter):
        self._c(lib().muca_run_graph(self._ctx, n_iters, sweeps_per_iter))

    def set_recursion(self, kind):
        """Weight recursion of every group: REC_PLAIN or REC_ACCUMULATED."""
        self._c(lib().muca_set_recursion(self._ctx, int(kind)))

    def get_flatness(self, g):
        """(min H / mean H, max H / mean H, bins hit) of the histogram merged
        by the last weight update of group g, over its active window."""
        out = np.zeros(3)
        self._c(lib().muca_get_flatness(self._ctx, g, _np_ptr(out)))
        return out

    def set_window(self, g, lo, hi, grow_flat=0.0, grow_step=0):
        """Active E_Delta window [lo, hi] of group g, growing by grow_step bins
        on each side after an iteration whose histogram has min H / mean H >=
        grow_flat over it (``muca_set_window``; grow_flat = 0: fixed)."""
        self._c(lib().muca_set_window(self._ctx, g, int(lo), int(hi), float(grow_flat),
                                      int(grow_step)))

    def set_bonds(self, g, J, jmax=None):
        """Couplings per bond of group g (``muca_set_bonds``): J int8
        [L^3][3] (forward x, y, z bonds), |J| <= jmax (default: the largest
        |J|, at least 1); None returns the group to the clean model."""
        if J is None:
            self._c(lib().muca_set_bonds(self._ctx, g, None, 0))
            return
        a = np.ascontiguousarray(J, dtype=np.int8).reshape(self.specs[g]["V"], 3)
        if jmax is None:
            jmax = max(1, int(np.abs(a.astype(np.int64)).max()))
        self._c(lib().muca_set_bonds(self._ctx, g, _np_ptr(a), int(jmax)))

    def get_window(self, g):
        out = np.zeros(2, dtype=np.int32)
        self._c(lib().muca_get_window(self._ctx, g, _np_ptr(out)))
        return int(out[0]), int(out[1])

    def walker_range(self, g):
        """(min, max) of the current E_Delta of group g's walkers."""
        tal = np.zeros((self.specs[g]["n_walkers"], 3), dtype=np.int32)
        self._c(lib().muca_get_state(self._ctx, g, None, _np_ptr(tal)))
        return int(tal[:, 1].min()), int(tal[:, 1].max())

    def iterate(self, max_iters, sweeps_per_iter, flat_min):
        """Weight iterations until every group's min H / mean H >= flat_min
        over a window that is its whole [e_min, e_max] (at most max_iters);
        returns the number of iterations run."""
        n = ctypes.c_int32(0)
        self._c(lib().muca_iterate(self._ctx, int(max_iters), int(sweeps_per_iter),
                                   float(flat_min), ctypes.byref(n)))
        return n.value

    def sync(self):
        self._c(lib().muca_sync(self._ctx))

    # -- time series
    def reserve_timeseries(self, n_samples):
        self._c(lib().muca_reserve_timeseries(self._ctx, n_samples))

    def timeseries_device(self, g):
        p = ctypes.c_void_p()
        n = ctypes.c_int64()
        self._c(lib().muca_timeseries_device(self._ctx, g, ctypes.byref(p), ctypes.byref(n)))
        return p.value, n.value

    def get_timeseries(self, g):
        _, n = self.timeseries_device(g)
        out = np.zeros((n, 3, self.specs[g]["n_walkers"]), dtype=np.int32)
        if n:
            self._c(lib().muca_get_timeseries(self._ctx, g, _np_ptr(out)))
        return out

    # -- inspection
    def sweep_count(self, g=0):
        v = ctypes.c_uint64()
        self._c(lib().muca_get_sweep_count(self._ctx, g, ctypes.byref(v)))
        return v.value

    def get_lnW(self, g):
        out = np.zeros(self.n_e(g))
        self._c(lib().muca_get_lnW(self._ctx, g, _np_ptr(out)))
        return out

    def set_lnW(self, g, lnW):
        a = np.ascontiguousarray(lnW, dtype=np.float64)
        assert a.shape == (self.n_e(g),)
        self._c(lib().muca_set_lnW(self._ctx, g, _np_ptr(a)))

    def get_table(self, g):
        out = np.zeros((self.n_e(g), 3, NK), dtype=np.uint32)
        self._c(lib().muca_get_table(self._ctx, g, _np_ptr(out)))
        return out

    def set_table(self, g, thr):
        a = np.ascontiguousarray(thr, dtype=np.uint32)
        assert a.shape == (self.n_e(g), 3, NK)
        self._c(lib().muca_set_table(self._ctx, g, _np_ptr(a)))

    def get_hist(self, g):
        out = np.zeros(self.n_e(g), dtype=np.uint64)
        self._c(lib().muca_get_hist(self._ctx, g, _np_ptr(out)))
        return out

    def set_hist(self, g, h):
        a = np.ascontiguousarray(h, dtype=np.uint64)
        assert a.shape == (self.n_e(g),)
        self._c(lib().muca_set_hist(self._ctx, g, _np_ptr(a)))

    def get_hist_device(self, g, out):
        """Copy group g's histogram into a CUDA tensor of n_e 64-bit integers."""
        assert out.is_cuda and out.numel() == self.n_e(g) and out.element_size() == 8
        self._c(lib().muca_get_hist_device(self._ctx, g, ctypes.c_void_p(out.data_ptr())))

    def set_hist_device(self, g, t):
        """Replace group g's histogram by a CUDA tensor of n_e 64-bit integers
        (complete on the device when called)."""
        assert t.is_cuda and t.numel() == self.n_e(g) and t.element_size() == 8
        self._c(lib().muca_set_hist_device(self._ctx, g, ctypes.c_void_p(t.data_ptr())))

    def get_state(self, g):
        self.n_e(g)
        s = self.specs[g]
        spins = np.zeros((s["n_walkers"], s["V"]), dtype=np.int8)
        tal = np.zeros((s["n_walkers"], 3), dtype=np.int32)
        self._c(lib().muca_get_state(self._ctx, g, _np_ptr(spins), _np_ptr(tal)))
        return spins, tal

    def set_state(self, g, spins):
        s = self.specs[g]
        a = np.ascontiguousarray(spins, dtype=np.int8)
        assert a.shape == (s["n_walkers"], s["V"])
        self._c(lib().muca_set_state(self._ctx, g, _np_ptr(a)))

    def check_tallies(self):
        self._c(lib().muca_check_tallies(self._ctx))

    def get_config(self, g):
        """(residency, walkers per block, lanes per walker) of group g."""
        r = ctypes.c_int32()
        w = ctypes.c_int32()
        p = ctypes.c_int32()
        self._c(lib().muca_get_config(self._ctx, g, ctypes.byref(r), ctypes.byref(w),
                                      ctypes.byref(p)))
        return r.value, w.value, p.value

    def checkpoint(self, path):
        self._c(lib().muca_checkpoint(self._ctx, os.fsencode(path)))

    def restore(self, path):
        self._c(lib().muca_restore(self._ctx, os.fsencode(path)))


def reweight(e_j, e_d, m, lnW, e_min, beta, V, delta_grid, precision=64, n_rows=None,
             row_len=None, row_stride=None, stream=None, no_alloc=False):
    """``muca_reweight`` (``muca_reweight_noalloc`` with no_alloc=True): e_j, e_d,
    m are torch int32 CUDA tensors (or raw device addresses with
    n_rows/row_len/row_stride given).  Returns numpy [n_grid][5]:
    <E_J>, <E_Delta>, C, chi, U4."""
    L = lib()
    ptrs = []
    for t in (e_j, e_d, m):
        if isinstance(t, int):
            ptrs.append(ctypes.c_void_p(t))
        else:
            import torch
            assert t.is_cuda and t.dtype == torch.int32, "samples must be int32 CUDA tensors"
            assert t.is_contiguous()
            ptrs.append(ctypes.c_void_p(t.data_ptr()))
    if n_rows is None:
        n_rows, row_len, row_stride = 1, int(e_d.numel()), int(e_d.numel())
    lnW = np.ascontiguousarray(lnW, dtype=np.float64)
    grid = np.ascontiguousarray(delta_grid, dtype=np.float64)
    out = np.zeros((len(grid), 5))
    fn = L.muca_reweight_noalloc if no_alloc else L.muca_reweight
    rc = fn(ptrs[0], ptrs[1], ptrs[2], n_rows, row_len, row_stride, _np_ptr(lnW), e_min,
            len(lnW), beta, V, _np_ptr(grid), len(grid), precision, _np_ptr(out),
            _stream_ptr(stream))
    _ck(rc)
    return out


def find_peak(e_j, e_d, lnW, e_min, beta, delta_lo, delta_hi, n_iter=60, n_jack=0, n_rows=None,
              row_len=None, row_stride=None, stream=None):
    """``muca_find_peak``: Delta*_L and C*_L (Sec. III) with jackknife errors.
    e_j, e_d are int32 CUDA tensors shaped [n_rows][row_len] (one row per
    sweep), or raw device addresses with n_rows/row_len/row_stride given.
    Returns (delta_star, delta_err, c_star, c_err, subsets [n_jack][2])."""
    ptrs = []
    for t in (e_j, e_d):
        if isinstance(t, int):
            ptrs.append(ctypes.c_void_p(t))
        else:
            import torch
            assert t.is_cuda and t.dtype == torch.int32, "samples must be int32 CUDA tensors"
            assert t.is_contiguous()
            ptrs.append(ctypes.c_void_p(t.data_ptr()))
    if n_rows is None:
        if e_d.dim() == 2:
            n_rows, row_len = int(e_d.shape[0]), int(e_d.shape[1])
        else:
            n_rows, row_len = 1, int(e_d.numel())
        row_stride = row_len
    lnW = np.ascontiguousarray(lnW, dtype=np.float64)
    out = np.zeros(4 + 2 * n_jack)
    _ck(lib().muca_find_peak(ptrs[0], ptrs[1], n_rows, row_len, row_stride, _np_ptr(lnW), e_min,
                             len(lnW), beta, delta_lo, delta_hi, n_iter, n_jack, _np_ptr(out),
                             _stream_ptr(stream)))
    return out[0], out[1], out[2], out[3], out[4:].reshape(n_jack, 2)


def equal_height(e_d, lnW, e_min, beta, split, delta_lo, delta_hi, n_iter=60, n_jack=0,
                 n_rows=None, row_len=None, row_stride=None, stream=None):
    """``muca_equal_height``: Delta_eqh and the barrier B with jackknife errors.
    e_d is an int32 CUDA tensor [n_rows][row_len] (or a raw device address with
    n_rows/row_len/row_stride given).  Returns (delta_eqh, delta_err, B, B_err,
    (E_lower_peak, E_upper_peak, E_min), subsets [n_jack][2])."""
    if isinstance(e_d, int):
        ptr = ctypes.c_void_p(e_d)
    else:
        import torch
        assert e_d.is_cuda and e_d.dtype == torch.int32, "samples must be int32 CUDA tensors"
        assert e_d.is_contiguous()
        ptr = ctypes.c_void_p(e_d.data_ptr())
    if n_rows is None:
        if e_d.dim() == 2:
            n_rows, row_len = int(e_d.shape[0]), int(e_d.shape[1])
        else:
            n_rows, row_len = 1, int(e_d.numel())
        row_stride = row_len
    lnW = np.ascontiguousarray(lnW, dtype=np.float64)
    out = np.zeros(7 + 2 * n_jack)
    _ck(lib().muca_equal_height(ptr, n_rows, row_len, row_stride, _np_ptr(lnW), e_min, len(lnW),
                                beta, split, delta_lo, delta_hi, n_iter, n_jack, _np_ptr(out),
                                _stream_ptr(stream)))
    return out[0], out[1], out[2], out[3], tuple(int(v) for v in out[4:7]), out[7:].reshape(n_jack, 2)


def reweight_context(ctx, g, delta_grid, precision=64, stream=None):
    """Reweight group g's recorded series with its current lnW."""
    s = ctx.specs[g]
    base, n = ctx.timeseries_device(g)
    W = s["n_walkers"]
    return reweight(base, base + 4 * W, base + 8 * W, ctx.get_lnW(g), s["e_min"], 1.0 / s["T"],
                    s["V"], delta_grid, precision, n_rows=n, row_len=W, row_stride=3 * W,
                    stream=stream)
