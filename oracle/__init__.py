"""CPU FP64 oracle for boxcar single-pulse detection (arXiv:1910.08324).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product library
(``paper_1910_08324_gb300``) never imports it, and this package never imports
the product: the two share no code.  The only module both sides use is the
seeded input generator ``spd_synth``, which holds none of the method's
arithmetic.

The arithmetic lives in ``spd_oracle.c`` (plain C, double precision, OpenMP over
DM rows); this module compiles it with gcc on first use and wraps it with
ctypes.  ``brute_search`` is a pure-Python restatement of the definition for
tiny inputs (Eq. boxcar, Eq. SNRlong, Eq. whitenoise, Eq. MSD03), used to pin
the C code.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spd_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libspd_oracle.so")
_lock = threading.Lock()
_lib = None

_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile ``spd_oracle.c`` into ``oracle/_build/libspd_oracle.so`` (gcc, -O2, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-fvisibility=hidden", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        i32, i64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        lib.spdo_grid_exhaustive.argtypes = [i32, _i32p, _i32p, i32]
        lib.spdo_grid_exhaustive.restype = i32
        lib.spdo_grid_boxdit.argtypes = [i32, i32, i32, _i32p, _i32p, i32]
        lib.spdo_grid_boxdit.restype = i32
        lib.spdo_grid_boxdit_iters.argtypes = [_i32p, i32, i32, i32, _i32p, _i32p, i32]
        lib.spdo_grid_boxdit_iters.restype = i32
        lib.spdo_grid_igrid.argtypes = [i32, i32, i32, _i32p, _i32p, i32]
        lib.spdo_grid_igrid.restype = i32
        lib.spdo_search.argtypes = [_f64p, i64, i64, i64, _i32p, _i32p, i32, i32,
                                    _f64p, _f64p, i32, i32, _f64p, _i32p, _f64p]
        lib.spdo_search.restype = i32
        lib.spdo_boxdit_steps.argtypes = [_f64p, i64, i64, i64, i32, i32, i32,
                                          _f64p, _f64p, _f64p, _i32p]
        lib.spdo_boxdit_steps.restype = i32
        lib.spdo_boxdit_steps_iters.argtypes = [_f64p, i64, i64, i64, _i32p, i32, i32, i32,
                                                _f64p, _f64p, _f64p, _i32p]
        lib.spdo_boxdit_steps_iters.restype = i32
        lib.spdo_igrid_steps.argtypes = [_f64p, i64, i64, i64, i32, i32, i32,
                                         _f64p, _f64p, _f64p, _i32p]
        lib.spdo_igrid_steps.restype = i32
        lib.spdo_rsnr_bounds.argtypes = [_i32p, _i32p, i32, i32, f64,
                                         ctypes.POINTER(f64), ctypes.POINTER(f64)]
        lib.spdo_rsnr_bounds.restype = None
        lib.spdo_pulse_rsnr.argtypes = [_i32p, _i32p, i32, i64, i32, i64, f64,
                                        ctypes.POINTER(i32)]
        lib.spdo_pulse_rsnr.restype = f64
        lib.spdo_sliding.argtypes = [_i32p, _i32p, i32, i32, i64, f64,
                                     ctypes.POINTER(f64), ctypes.POINTER(f64),
                                     ctypes.POINTER(f64)]
        lib.spdo_sliding.restype = None
        lib.spdo_msd_levels.argtypes = [_f64p, i64, i64, i64, i32, f64, i32, _f64p, _f64p, _i64p]
        lib.spdo_msd_levels.restype = ctypes.c_int
        lib.spdo_msd_table.argtypes = [_f64p, _f64p, _i64p, i64, i32, _i32p, i32, _f64p, _f64p]
        lib.spdo_msd_table.restype = ctypes.c_int
        lib.spdo_candidates.argtypes = [_f64p, ctypes.c_void_p, i64, i64, f64, i32,
                                        _i64p, _i64p, _i32p, _f64p, i64]
        lib.spdo_candidates.restype = i64
        _lib = lib
        return lib


# --------------------------------------------------------------------------- grids
class Grid:
    """A width table: ascending widths ``L`` and their separations ``Ls`` (int32)."""

    def __init__(self, L, Ls):
        self.L = np.ascontiguousarray(L, dtype=np.int32)
        self.Ls = np.ascontiguousarray(Ls, dtype=np.int32)

    def __len__(self):
        return int(self.L.size)

    def __repr__(self):
        return "Grid(n=%d, L_end=%d)" % (len(self), int(self.L[-1]))


def _grid_call(fn, *args, cap=1 << 16):
    L = np.zeros(cap, np.int32)
    Ls = np.zeros(cap, np.int32)
    n = fn(*args, L, Ls, cap)
    if n < 0:
        raise ValueError("oracle grid builder rejected the parameters (code %d)" % n)
    return Grid(L[:n].copy(), Ls[:n].copy())


def grid_exhaustive(lmax: int) -> Grid:
    """Every width 1..lmax at every sample (the ideal SPD of Sec. 3.1)."""
    return _grid_call(_load().spdo_grid_exhaustive, int(lmax))


def _klist(k):
    ks = np.atleast_1d(np.asarray(k, np.int32)).ravel()
    return np.ascontiguousarray(ks), int(ks.size)


def grid_boxdit(k, s_end: int, n_iter: int = 0) -> Grid:
    """BoxDIT, D = 2 (Alg. 1); stops at the first width >= s_end.

    ``k`` is L^i_max: one even number for every iteration, or a sequence with
    one per iteration (Sec. 3.1: it may change from iteration to iteration),
    whose last entry repeats for later iterations.
    """
    ks, nk = _klist(k)
    return _grid_call(_load().spdo_grid_boxdit_iters, ks, nk, int(s_end), int(n_iter))


def grid_igrid(d: int, P: int, s_end: int) -> Grid:
    """IGRID IG(d) with P layers per step (Sec. 3.2, Eq. boxcarsize, Table 1)."""
    return _grid_call(_load().spdo_grid_igrid, int(d), int(P), int(s_end))


# --------------------------------------------------------------------------- search
def _rows(x):
    x = np.asarray(x)
    if x.ndim == 1:
        x = x[None, :]
    return np.ascontiguousarray(x, dtype=np.float64)


def _noise_arrays(ndm, mu, sigma, n_grid=None, mode=0):
    if mode == 0:
        mu = np.broadcast_to(np.asarray(mu, np.float64), (ndm,))
        sigma = np.broadcast_to(np.asarray(sigma, np.float64), (ndm,))
    else:
        mu = np.asarray(mu, np.float64).reshape(ndm, n_grid)
        sigma = np.asarray(sigma, np.float64).reshape(ndm, n_grid)
    return np.ascontiguousarray(mu), np.ascontiguousarray(sigma)


def search(x, grid: Grid, mu=0.0, sigma=1.0, noise_mode: int = 0, literal: bool = False,
           threads: int = 0):
    """Definition-form search (O1).  Returns ``(Y, W, Y2)`` as dense [ndm, nt] arrays.

    ``W`` is the index into ``grid`` of the smallest width reaching the maximum;
    ``Y2`` is the best SNR among the other eligible widths.
    """
    x = _rows(x)
    ndm, nt = x.shape
    mu, sigma = _noise_arrays(ndm, mu, sigma, len(grid), noise_mode)
    Y = np.empty((ndm, nt), np.float64)
    W = np.empty((ndm, nt), np.int32)
    Y2 = np.empty((ndm, nt), np.float64)
    rc = _load().spdo_search(x.reshape(-1), ndm, nt, nt, grid.L, grid.Ls, len(grid),
                             int(noise_mode), mu.reshape(-1), sigma.reshape(-1),
                             int(bool(literal)), int(threads), Y.reshape(-1),
                             W.reshape(-1), Y2.reshape(-1))
    if rc != 0:
        raise RuntimeError("spdo_search failed (%d)" % rc)
    return Y, W, Y2


def boxdit_steps(x, k, s_end: int, mu=0.0, sigma=1.0, n_iter: int = 0):
    """Alg. 1 run literally (O2).  Returns ``(Y, Wlen)``; ``Wlen`` holds widths.

    ``k``: L^i_max, one even number or one per iteration (as in grid_boxdit).
    """
    x = _rows(x)
    ndm, nt = x.shape
    mu, sigma = _noise_arrays(ndm, mu, sigma)
    Y = np.empty((ndm, nt), np.float64)
    Wl = np.empty((ndm, nt), np.int32)
    ks, nk = _klist(k)
    rc = _load().spdo_boxdit_steps_iters(x.reshape(-1), ndm, nt, nt, ks, nk, int(s_end),
                                         int(n_iter), mu, sigma, Y.reshape(-1), Wl.reshape(-1))
    if rc != 0:
        raise RuntimeError("spdo_boxdit_steps failed (%d)" % rc)
    return Y, Wl


def igrid_steps(x, d: int, P: int, s_end: int, mu=0.0, sigma=1.0):
    """The IGRID layer tree of Sec. 3.2 run literally (O2).  Returns ``(Y, Wlen)``."""
    x = _rows(x)
    ndm, nt = x.shape
    mu, sigma = _noise_arrays(ndm, mu, sigma)
    Y = np.empty((ndm, nt), np.float64)
    Wl = np.empty((ndm, nt), np.int32)
    rc = _load().spdo_igrid_steps(x.reshape(-1), ndm, nt, nt, int(d), int(P), int(s_end),
                                  mu, sigma, Y.reshape(-1), Wl.reshape(-1))
    if rc != 0:
        raise RuntimeError("spdo_igrid_steps failed (%d)" % rc)
    return Y, Wl


# --------------------------------------------------------------------------- bounds
def rsnr_bounds(grid: Grid, S: int, C: float = 1.0):
    """Appendix A: ``(RSNR_max(S), RSNR_min(S))`` (Eq. RSNRmax, Eq. RSNRmin)."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _load().spdo_rsnr_bounds(grid.L, grid.Ls, len(grid), int(S), float(C),
                             ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def pulse_rsnr(grid: Grid, nt: int, S: int, t: int, C: float = 1.0):
    """RSNR of one noise-free rectangular pulse [t, t+S) (Eq. RSNR).  Returns (rsnr, L)."""
    bl = ctypes.c_int32()
    v = _load().spdo_pulse_rsnr(grid.L, grid.Ls, len(grid), int(nt), int(S), int(t),
                                float(C), ctypes.byref(bl))
    return v, bl.value


def sliding(grid: Grid, S: int, n_shift: int, C: float = 1.0):
    """Sec. 4.1 sliding-pulse measurement: ``(max, min, mean)`` RSNR over shifts."""
    a, b, m = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _load().spdo_sliding(grid.L, grid.Ls, len(grid), int(S), int(n_shift), float(C),
                         ctypes.byref(a), ctypes.byref(b), ctypes.byref(m))
    return a.value, b.value, m.value


# --------------------------------------------------------------------------- peaks
def candidates(Y, W=None, thr: float = 6.0, R: int = 1, cap: int | None = None):
    """Threshold + local-maximum candidates, ordered by (row, start).

    Returns ``(total, rows, starts, widx, snr)`` where the arrays hold the first
    ``cap`` records.
    """
    Y = _rows(Y)
    ndm, nt = Y.shape
    if cap is None:
        cap = int(np.count_nonzero(Y >= thr))
    cap = max(int(cap), 1)
    Wp = None
    if W is not None:
        W = np.ascontiguousarray(np.asarray(W, np.int32).reshape(ndm, nt))
        Wp = W.ctypes.data
    rows = np.zeros(cap, np.int64)
    starts = np.zeros(cap, np.int64)
    widx = np.zeros(cap, np.int32)
    snr = np.zeros(cap, np.float64)
    n = _load().spdo_candidates(Y.reshape(-1), Wp, ndm, nt, float(thr), int(R), rows,
                                starts, widx, snr, cap)
    k = min(n, cap)
    return int(n), rows[:k], starts[:k], widx[:k], snr[:k]


# --------------------------------------------------------------------------- brute force
def brute_search(x, L, Ls, mu=0.0, sigma=1.0):
    """Pure-Python restatement of the definition for tiny inputs (one row).

    Loops over every start s and every width, sums the boxcar sample by sample
    (Eq. boxcar), normalises with the white-noise statistics (Eq. SNRlong and
    Eq. whitenoise) and keeps the largest SNR, first width on ties (Eq. MSD03).
    """
    x = [float(v) for v in np.asarray(x, np.float64).ravel()]
    nt = len(x)
    Y, W = [], []
    for s in range(nt):
        best, bi = -math.inf, -1
        for g, (w, sep) in enumerate(zip(L, Ls)):
            if s % sep or s + w > nt:
                continue
            tot = 0.0
            for j in range(w):
                tot += x[s + j]
            snr = (tot - w * mu) / (math.sqrt(w) * sigma)
            if snr > best:
                best, bi = snr, g
        Y.append(best)
        W.append(bi)
    return np.array(Y), np.array(W, np.int32)


def msd_levels(x, nlev: int, thr: float = 2.0, max_passes: int = 10):
    """Mean, deviation and count of every row at decimations 2^0..2^(nlev-1), with
    iterated outlier rejection at ``thr`` deviations (thr <= 0: none).
    Returns ``(mu, sigma, n)``, each [ndm, nlev]."""
    x = _rows(x)
    ndm, nt = x.shape
    mu = np.empty((ndm, nlev), np.float64)
    sg = np.empty((ndm, nlev), np.float64)
    n = np.empty((ndm, nlev), np.int64)
    rc = _load().spdo_msd_levels(x.reshape(-1), ndm, nt, nt, int(nlev), float(thr),
                                 int(max_passes), mu.reshape(-1), sg.reshape(-1), n.reshape(-1))
    if rc != 0:
        raise RuntimeError("spdo_msd_levels failed (%d)" % rc)
    return mu, sg, n


def msd_table(mu, sigma, n, widths):
    """Per-width table (mu_L, sigma_L), each [ndm, len(widths)], from msd_levels."""
    mu = np.ascontiguousarray(mu, np.float64)
    sg = np.ascontiguousarray(sigma, np.float64)
    n = np.ascontiguousarray(n, np.int64)
    ndm, nlev = mu.shape
    L = np.ascontiguousarray(widths, np.int32)
    tm = np.empty((ndm, len(L)), np.float64)
    ts = np.empty((ndm, len(L)), np.float64)
    rc = _load().spdo_msd_table(mu.reshape(-1), sg.reshape(-1), n.reshape(-1), ndm, nlev, L,
                                len(L), tm.reshape(-1), ts.reshape(-1))
    if rc != 0:
        raise RuntimeError("spdo_msd_table failed (%d)" % rc)
    return tm, ts
