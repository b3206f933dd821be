"""ctypes binding of libspd.so (argument marshalling only).

The C ABI (``include/spd.h``) takes plain device pointers and a CUDA stream
handle.  The ``spd_*`` functions here mirror it one to one and accept integer
pointers; ``execute``/``candidates``/``search`` accept torch tensors and use the
current torch stream.  Errors raise ``SpdError`` carrying the status code.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

SPD_ALGO_EXHAUSTIVE, SPD_ALGO_BOXDIT, SPD_ALGO_IGRID = 0, 1, 2
SPD_F32, SPD_F16, SPD_BF16, SPD_U8 = 0, 1, 2, 3

_STATUS = {0: "SPD_OK", 1: "SPD_ERR_INVALID_ARG", 2: "SPD_ERR_UNSUPPORTED", 3: "SPD_ERR_CUDA",
           4: "SPD_ERR_WORKSPACE_TOO_SMALL", 5: "SPD_ERR_BUFFER_TOO_SMALL", 6: "SPD_ERR_TIMEOUT",
           7: "SPD_ERR_HOST_ALLOC"}

# struct spd_candidate {int32 row; int32 width_idx; int64 start; float snr; int32 width;}
CANDIDATE_DTYPE = np.dtype([("row", np.int32), ("width_idx", np.int32), ("start", np.int64),
                            ("snr", np.float32), ("width", np.int32)])
assert CANDIDATE_DTYPE.itemsize == 24


class SpdError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__("%s: %s (%s)" % (where, _STATUS.get(status, status),
                                          spd_status_string(status)))


class _Desc(ctypes.Structure):
    _fields_ = [("algo", ctypes.c_int32), ("dtype", ctypes.c_int32), ("s_end", ctypes.c_int32),
                ("boxdit_lmax", ctypes.c_int32), ("igrid_depth", ctypes.c_int32),
                ("igrid_layers", ctypes.c_int32), ("ndm", ctypes.c_int64), ("nt", ctypes.c_int64),
                ("ld", ctypes.c_int64)]


class _Noise(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("mu", ctypes.c_void_p), ("sigma", ctypes.c_void_p)]


class _RangeIO(ctypes.Structure):
    _fields_ = [("d_x", ctypes.c_void_p), ("d_snr", ctypes.c_void_p), ("d_width_idx", ctypes.c_void_p),
                ("d_mu", ctypes.c_void_p), ("d_sigma", ctypes.c_void_p), ("d_ready", ctypes.c_void_p)]


_lib = None
_lock = threading.Lock()
_SYMBOLS = ["spd_status_string", "spd_version", "spd_plan_create", "spd_plan_destroy",
            "spd_plan_widths", "spd_workspace_size", "spd_execute", "spd_candidates",
            "spd_search", "spd_sync_status", "spd_candidates_static", "spd_noise_stats",
            "spd_plan_set_segment", "spd_batch_create", "spd_batch_destroy", "spd_batch_set_segment",
            "spd_batch_set_wait_ns", "spd_batch_set_ctas_per_sm", "spd_batch_workspace_size", "spd_batch_execute", "spd_batch_status",
            "spd_batch_candidates", "spd_net_decimate", "spd_net_forward", "spd_net_gradient",
            "spd_net_adam", "spd_net_select", "spd_net_gather", "spd_plan_set_starts", "spd_plan_create_grid",
            "spd_net_gradient_ordered", "spd_candidates_status", "spd_plan_create_boxdit",
            "spd_proposal_create", "spd_proposal_destroy", "spd_proposal_workspace_size",
            "spd_proposal_widths", "spd_propose_search", "spd_search_blocks"]


def library_path() -> str:
    return _build.LIB


def load_library():
    """Load libspd.so, building it first if it is missing or stale (needs nvcc)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build()
        lib = ctypes.CDLL(path)
        vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
        lib.spd_status_string.argtypes = [ctypes.c_int]
        lib.spd_status_string.restype = ctypes.c_char_p
        lib.spd_version.argtypes = []
        lib.spd_version.restype = ctypes.c_char_p
        lib.spd_plan_create.argtypes = [ctypes.POINTER(_Desc), ctypes.POINTER(vp)]
        lib.spd_plan_destroy.argtypes = [vp]
        lib.spd_plan_widths.argtypes = [vp, vp, vp, i32, ctypes.POINTER(i32)]
        lib.spd_workspace_size.argtypes = [vp, ctypes.POINTER(sz)]
        lib.spd_execute.argtypes = [vp, vp, ctypes.POINTER(_Noise), vp, vp, vp, sz, vp]
        lib.spd_candidates.argtypes = [vp, vp, vp, ctypes.c_float, i32, vp, i64, vp, vp, sz, i32, vp]
        lib.spd_search.argtypes = [vp, vp, ctypes.POINTER(_Noise), vp, vp, ctypes.c_float, i32, vp,
                                   i64, vp, vp, sz, vp]
        lib.spd_sync_status.argtypes = [vp, vp]
        lib.spd_candidates_static.argtypes = [vp, vp, vp, ctypes.c_float, i32, vp, i64, vp, vp]
        lib.spd_candidates_status.argtypes = [vp, i64, ctypes.POINTER(i64), vp]
        lib.spd_noise_stats.argtypes = [vp, vp, ctypes.c_float, i32, vp, vp, vp, sz, vp]
        lib.spd_plan_set_segment.argtypes = [vp, i32]
        lib.spd_plan_set_starts.argtypes = [vp, i64]
        lib.spd_plan_create_grid.argtypes = [ctypes.POINTER(_Desc), vp, vp, i32, ctypes.POINTER(vp)]
        lib.spd_plan_create_boxdit.argtypes = [ctypes.POINTER(_Desc), vp, i32, i32, ctypes.POINTER(vp)]
        lib.spd_proposal_create.argtypes = [ctypes.POINTER(_Desc), i32, ctypes.c_int64, ctypes.POINTER(vp)]
        lib.spd_proposal_destroy.argtypes = [vp]
        lib.spd_proposal_workspace_size.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
        lib.spd_proposal_widths.argtypes = [vp, vp, vp, i32, ctypes.POINTER(i32)]
        lib.spd_propose_search.argtypes = [vp, vp, vp, ctypes.POINTER(_Noise), ctypes.c_float, ctypes.c_float,
                                           vp, ctypes.c_int64, vp, ctypes.POINTER(ctypes.c_int64), vp,
                                           ctypes.c_size_t, vp]
        lib.spd_search_blocks.argtypes = [vp, vp, ctypes.POINTER(_Noise), vp, ctypes.c_int64, ctypes.c_float,
                                          vp, ctypes.c_int64, vp, vp, ctypes.c_size_t, vp]
        lib.spd_net_param_count.argtypes = []
        lib.spd_net_param_count.restype = ctypes.c_int32
        lib.spd_net_decimate.argtypes = [vp, i32, i64, i64, i64, vp, vp, vp, vp]
        lib.spd_net_forward.argtypes = [vp, vp, i64, vp, vp]
        lib.spd_net_gradient.argtypes = [vp, vp, vp, i64, vp, vp, vp]
        lib.spd_net_adam.argtypes = [vp, vp, vp, vp, i64, ctypes.c_float, i32, vp]
        lib.spd_net_gradient_workspace_size.argtypes = []
        lib.spd_net_gradient_workspace_size.restype = sz
        lib.spd_net_gradient_ordered.argtypes = [vp, vp, vp, i64, vp, vp, vp, sz, vp]
        lib.spd_net_select.argtypes = [vp, i64, ctypes.c_float, vp, i64, vp, vp]
        lib.spd_net_gather.argtypes = [vp, i32, i64, i64, i64, vp, i64, i32, i32, i32, vp, i64, vp]
        lib.spd_batch_create.argtypes = [ctypes.POINTER(_Desc), vp, vp, vp, i32, ctypes.POINTER(vp)]
        lib.spd_batch_destroy.argtypes = [vp]
        lib.spd_batch_set_segment.argtypes = [vp, i32]
        lib.spd_batch_set_wait_ns.argtypes = [vp, i64]
        lib.spd_batch_set_ctas_per_sm.argtypes = [vp, i32]
        lib.spd_batch_workspace_size.argtypes = [vp, ctypes.POINTER(sz)]
        lib.spd_batch_execute.argtypes = [vp, ctypes.POINTER(_RangeIO), vp, sz, vp]
        lib.spd_batch_status.argtypes = [vp, vp, vp]
        lib.spd_batch_candidates.argtypes = [vp, i32, vp, vp, ctypes.c_float, i32, vp, i64, vp, vp, sz,
                                             i32, vp]
        for name in _SYMBOLS[2:]:
            getattr(lib, name).restype = ctypes.c_int
        _lib = lib
        return lib


def _check(status: int, where: str):
    if status != 0:
        raise SpdError(status, where)


def spd_status_string(status: int) -> str:
    return load_library().spd_status_string(int(status)).decode()


def spd_version() -> str:
    return load_library().spd_version().decode()


class Plan:
    """Owns an ``spd_plan*``; destroyed with the object."""

    def __init__(self, handle: int, desc: _Desc):
        self.handle = handle
        self.desc = desc
        self.ndm, self.nt, self.ld = int(desc.ndm), int(desc.nt), int(desc.ld)

    def widths(self):
        return spd_plan_widths(self)

    def workspace_size(self) -> int:
        return spd_workspace_size(self)

    def close(self):
        if self.handle:
            spd_plan_destroy(self)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def spd_plan_create(algo: int, s_end: int, ndm: int, nt: int, ld: int | None = None,
                    boxdit_lmax: int = 0, igrid_depth: int = 0, igrid_layers: int = 0,
                    dtype: int = SPD_F32) -> Plan:
    lib = load_library()
    d = _Desc(int(algo), int(dtype), int(s_end), int(boxdit_lmax), int(igrid_depth),
              int(igrid_layers), int(ndm), int(nt), int(nt if ld is None else ld))
    h = ctypes.c_void_p()
    _check(lib.spd_plan_create(ctypes.byref(d), ctypes.byref(h)), "spd_plan_create")
    return Plan(h.value, d)


class Proposal:
    """Owns an ``spd_proposal*`` (``spd_proposal_create``); destroyed with the object."""

    def __init__(self, handle: int, desc: _Desc, radius: int, max_blocks: int):
        self.handle = handle
        self.desc = desc
        self.radius = int(radius)
        self.max_blocks = int(max_blocks)
        self.ndm, self.nt, self.ld = int(desc.ndm), int(desc.nt), int(desc.ld)

    def workspace_size(self) -> int:
        n = ctypes.c_size_t()
        _check(load_library().spd_proposal_workspace_size(ctypes.c_void_p(self.handle), ctypes.byref(n)),
               "spd_proposal_workspace_size")
        return int(n.value)

    def widths(self):
        lib = load_library()
        n = ctypes.c_int32()
        h = ctypes.c_void_p(self.handle)
        _check(lib.spd_proposal_widths(h, None, None, 0, ctypes.byref(n)), "spd_proposal_widths")
        w = np.zeros(n.value, np.int32)
        sp = np.zeros(n.value, np.int32)
        _check(lib.spd_proposal_widths(h, w.ctypes.data, sp.ctypes.data, n.value, ctypes.byref(n)),
               "spd_proposal_widths")
        return w, sp

    def close(self):
        if self.handle:
            _check(load_library().spd_proposal_destroy(ctypes.c_void_p(self.handle)), "spd_proposal_destroy")
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def spd_proposal_create(algo: int, s_end: int, ndm: int, nt: int, ld: int | None = None, boxdit_lmax: int = 0,
                        igrid_depth: int = 0, igrid_layers: int = 0, dtype: int = SPD_F32, peak_radius: int = 1,
                        max_blocks: int = 1 << 16) -> Proposal:
    """A proposal search of [ndm, nt] series (nt a multiple of 4096) with the given grid."""
    lib = load_library()
    d = _Desc(int(algo), int(dtype), int(s_end), int(boxdit_lmax), int(igrid_depth),
              int(igrid_layers), int(ndm), int(nt), int(nt if ld is None else ld))
    h = ctypes.c_void_p()
    _check(lib.spd_proposal_create(ctypes.byref(d), int(peak_radius), int(max_blocks), ctypes.byref(h)),
           "spd_proposal_create")
    return Proposal(h.value, d, peak_radius, max_blocks)


def spd_propose_search(prop: Proposal, params: int, x: int, mu: int, sigma: int, logit_threshold: float,
                       threshold: float, out: int, cap: int, count: int, ws: int, ws_bytes: int, stream: int = 0,
                       noise_mode: int = 0) -> int:
    """Runs ``spd_propose_search``; returns the number of flagged blocks (raises
    SPD_ERR_BUFFER_TOO_SMALL when it exceeds the proposal's max_blocks)."""
    nz = _Noise(int(noise_mode), mu, sigma)
    nb = ctypes.c_int64(0)
    st = load_library().spd_propose_search(ctypes.c_void_p(prop.handle), params, x, ctypes.byref(nz),
                                           float(logit_threshold), float(threshold), out or None, int(cap),
                                           count, ctypes.byref(nb), ws, ws_bytes, stream or None)
    if st != 0:
        err = SpdError(st, "spd_propose_search")
        err.n_blocks = int(nb.value)  # the flagged blocks (when there were more than max_blocks)
        raise err
    return int(nb.value)


def spd_search_blocks(prop: Proposal, x: int, mu: int, sigma: int, ids: int, n_ids: int, threshold: float,
                      out: int, cap: int, count: int, ws: int, ws_bytes: int, stream: int = 0, noise_mode: int = 0):
    nz = _Noise(int(noise_mode), mu, sigma)
    _check(load_library().spd_search_blocks(ctypes.c_void_p(prop.handle), x, ctypes.byref(nz), ids or None,
                                            int(n_ids), float(threshold), out or None, int(cap), count, ws,
                                            ws_bytes, stream or None), "spd_search_blocks")


def spd_plan_create_boxdit(lmax, s_end: int, ndm: int, nt: int, ld: int | None = None, n_iter: int = 0,
                           dtype: int = SPD_F32) -> Plan:
    """BoxDIT plan with one maximum width L^i_max per iteration (``lmax``, a
    sequence of even values; the last repeats), up to the first width >= s_end,
    or exactly ``n_iter`` iterations when n_iter > 0."""
    lib = load_library()
    k = np.ascontiguousarray(np.atleast_1d(np.asarray(lmax, np.int32)).ravel())
    d = _Desc(SPD_ALGO_BOXDIT, int(dtype), int(s_end), int(k[0]) if k.size else 0, 0, 0, int(ndm), int(nt),
              int(nt if ld is None else ld))
    h = ctypes.c_void_p()
    _check(lib.spd_plan_create_boxdit(ctypes.byref(d), k.ctypes.data, int(k.size), int(n_iter), ctypes.byref(h)),
           "spd_plan_create_boxdit")
    return Plan(h.value, d)


def spd_plan_create_grid(widths, seps, ndm: int, nt: int, ld: int | None = None, dtype: int = SPD_F32) -> Plan:
    """Plan over an explicit width set: widths[i] searched at the starts that are
    multiples of seps[i] (width 1 at every start first; separations powers of two)."""
    lib = load_library()
    w = np.ascontiguousarray(np.asarray(widths, np.int32))
    s = np.ascontiguousarray(np.asarray(seps, np.int32))
    if w.shape != s.shape or w.ndim != 1:
        raise SpdError(1, "spd_plan_create_grid: widths and seps differ in shape")
    d = _Desc(SPD_ALGO_EXHAUSTIVE, int(dtype), int(w[-1]) if len(w) else 1, 0, 0, 0, int(ndm), int(nt),
              int(nt if ld is None else ld))
    h = ctypes.c_void_p()
    _check(lib.spd_plan_create_grid(ctypes.byref(d), w.ctypes.data, s.ctypes.data, len(w), ctypes.byref(h)),
           "spd_plan_create_grid")
    return Plan(h.value, d)


def spd_plan_destroy(plan: Plan):
    _check(load_library().spd_plan_destroy(ctypes.c_void_p(plan.handle)), "spd_plan_destroy")


def spd_plan_widths(plan: Plan):
    lib = load_library()
    n = ctypes.c_int32()
    _check(lib.spd_plan_widths(ctypes.c_void_p(plan.handle), None, None, 0, ctypes.byref(n)),
           "spd_plan_widths")
    w = np.zeros(n.value, np.int32)
    s = np.zeros(n.value, np.int32)
    _check(lib.spd_plan_widths(ctypes.c_void_p(plan.handle), w.ctypes.data, s.ctypes.data,
                               n.value, ctypes.byref(n)), "spd_plan_widths")
    return w, s


def spd_workspace_size(plan: Plan) -> int:
    b = ctypes.c_size_t()
    _check(load_library().spd_workspace_size(ctypes.c_void_p(plan.handle), ctypes.byref(b)),
           "spd_workspace_size")
    return int(b.value)


def spd_execute(plan: Plan, x: int, mu: int, sigma: int, snr: int, width_idx: int, ws: int,
                ws_bytes: int, stream: int = 0, noise_mode: int = 0):
    nz = _Noise(int(noise_mode), mu, sigma)
    _check(load_library().spd_execute(ctypes.c_void_p(plan.handle), x, ctypes.byref(nz), snr,
                                      width_idx, ws, ws_bytes, stream or None), "spd_execute")


def spd_candidates(plan: Plan, snr: int, width_idx: int, threshold: float, peak_radius: int,
                   out: int, cap: int, count: int, ws: int, ws_bytes: int, use_tile_max: int = 0,
                   stream: int = 0):
    _check(load_library().spd_candidates(ctypes.c_void_p(plan.handle), snr, width_idx,
                                         float(threshold), int(peak_radius), out or None,
                                         int(cap), count, ws, ws_bytes, int(use_tile_max),
                                         stream or None),
           "spd_candidates")


def spd_candidates_status(count: int, cap: int, stream: int = 0) -> int:
    """Waits for the stream and returns the true record count at device address
    ``count``; raises SpdError (SPD_ERR_BUFFER_TOO_SMALL) when it exceeds cap."""
    total = ctypes.c_int64(-1)
    _check(load_library().spd_candidates_status(count, int(cap), ctypes.byref(total), stream or None),
           "spd_candidates_status")
    return int(total.value)


def spd_candidates_static(plan: Plan, snr: int, width_idx: int, threshold: float,
                          peak_radius: int, out: int, cap: int, count: int, stream: int = 0):
    """spd_candidates with the library's own static scratch instead of a workspace."""
    _check(load_library().spd_candidates_static(ctypes.c_void_p(plan.handle), snr, width_idx,
                                                float(threshold), int(peak_radius), out or None,
                                                int(cap), count, stream or None),
           "spd_candidates_static")


def spd_search(plan: Plan, x: int, mu: int, sigma: int, snr: int, width_idx: int,
               threshold: float, peak_radius: int, out: int, cap: int, count: int, ws: int,
               ws_bytes: int, stream: int = 0, noise_mode: int = 0):
    nz = _Noise(int(noise_mode), mu, sigma)
    _check(load_library().spd_search(ctypes.c_void_p(plan.handle), x, ctypes.byref(nz), snr,
                                     width_idx, float(threshold), int(peak_radius), out or None,
                                     int(cap), count, ws, ws_bytes, stream or None), "spd_search")


def spd_noise_stats(plan: Plan, x: int, outlier_sigma: float, max_passes: int, mu: int, sigma: int,
                    ws: int, ws_bytes: int, stream: int = 0):
    _check(load_library().spd_noise_stats(ctypes.c_void_p(plan.handle), x, float(outlier_sigma),
                                          int(max_passes), mu, sigma, ws, ws_bytes, stream or None),
           "spd_noise_stats")


def spd_plan_set_starts(plan: Plan, n_starts: int):
    _check(load_library().spd_plan_set_starts(ctypes.c_void_p(plan.handle), int(n_starts)), "spd_plan_set_starts")


def spd_plan_set_segment(plan: Plan, segment: int):
    _check(load_library().spd_plan_set_segment(ctypes.c_void_p(plan.handle), int(segment)),
           "spd_plan_set_segment")


class Batch:
    """Owns an ``spd_batch*`` (ranges of one grid searched in one launch)."""

    def __init__(self, handle: int, ndm, nt, ld):
        self.handle = handle
        self.ndm, self.nt, self.ld = list(ndm), list(nt), list(ld)

    def close(self):
        if self.handle:
            load_library().spd_batch_destroy(ctypes.c_void_p(self.handle))
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def workspace_size(self) -> int:
        b = ctypes.c_size_t()
        _check(load_library().spd_batch_workspace_size(ctypes.c_void_p(self.handle), ctypes.byref(b)),
               "spd_batch_workspace_size")
        return int(b.value)

    def set_segment(self, segment: int):
        _check(load_library().spd_batch_set_segment(ctypes.c_void_p(self.handle), int(segment)),
               "spd_batch_set_segment")

    def set_ctas_per_sm(self, n: int):
        _check(load_library().spd_batch_set_ctas_per_sm(ctypes.c_void_p(self.handle), int(n)),
               "spd_batch_set_ctas_per_sm")

    def set_wait_ns(self, ns: int):
        _check(load_library().spd_batch_set_wait_ns(ctypes.c_void_p(self.handle), int(ns)),
               "spd_batch_set_wait_ns")


def spd_batch_create(algo: int, s_end: int, ndm, nt, ld=None, boxdit_lmax: int = 0,
                     igrid_depth: int = 0, igrid_layers: int = 0, dtype: int = SPD_F32) -> Batch:
    import numpy as np
    lib = load_library()
    d = _Desc(int(algo), int(dtype), int(s_end), int(boxdit_lmax), int(igrid_depth), int(igrid_layers), 1, 1, 1)
    n = len(ndm)
    a_ndm = np.ascontiguousarray(ndm, np.int64)
    a_nt = np.ascontiguousarray(nt, np.int64)
    a_ld = np.ascontiguousarray(nt if ld is None else ld, np.int64)
    h = ctypes.c_void_p()
    _check(lib.spd_batch_create(ctypes.byref(d), a_ndm.ctypes.data, a_nt.ctypes.data, a_ld.ctypes.data,
                                n, ctypes.byref(h)), "spd_batch_create")
    return Batch(h.value, a_ndm, a_nt, a_ld)


def _range_ios(xs, ys, ws_idx, mus, sigmas, readys):
    n = len(xs)
    arr = (_RangeIO * n)()
    for r in range(n):
        arr[r] = _RangeIO(xs[r], ys[r], ws_idx[r], mus[r], sigmas[r], (readys[r] if readys else 0) or None)
    return arr


def spd_batch_execute(batch: Batch, xs, ys, ws_idx, mus, sigmas, ws: int, ws_bytes: int, stream: int = 0,
                      readys=None):
    """xs, ys, ws_idx, mus, sigmas, readys: per-range device addresses (ints)."""
    arr = _range_ios(xs, ys, ws_idx, mus, sigmas, readys)
    _check(load_library().spd_batch_execute(ctypes.c_void_p(batch.handle), arr, ws, ws_bytes,
                                            stream or None), "spd_batch_execute")


def spd_batch_status(batch: Batch, ws: int, stream: int = 0):
    _check(load_library().spd_batch_status(ctypes.c_void_p(batch.handle), ws, stream or None),
           "spd_batch_status")


def spd_batch_candidates(batch: Batch, rng: int, snr: int, width_idx: int, threshold: float,
                         peak_radius: int, out: int, cap: int, count: int, ws: int, ws_bytes: int,
                         use_tile_max: int = 1, stream: int = 0):
    _check(load_library().spd_batch_candidates(ctypes.c_void_p(batch.handle), int(rng), snr, width_idx,
                                               float(threshold), int(peak_radius), out or None,
                                               int(cap), count, ws, ws_bytes, int(use_tile_max),
                                               stream or None), "spd_batch_candidates")


def spd_sync_status(plan: Plan, stream: int = 0):
    _check(load_library().spd_sync_status(ctypes.c_void_p(plan.handle), stream or None),
           "spd_sync_status")


# ----------------------------------------------------------------------------- torch helpers
def _stream(stream):
    import torch
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def _ptr(t):
    return 0 if t is None else int(t.data_ptr())


def _need(where: str, plan: Plan, **tensors):
    """Raise SPD_ERR_BUFFER_TOO_SMALL unless every given tensor is contiguous and
    holds the plan's ndm * ld elements (the C calls take bare pointers and
    cannot check this themselves)."""
    n = plan.ndm * plan.ld
    for name, t in tensors.items():
        if t is None:
            continue
        if not t.is_contiguous() or t.numel() < n:
            raise SpdError(5, "%s: %s needs %d contiguous elements ([ndm][ld] = [%d][%d]), got %s %s"
                           % (where, name, n, plan.ndm, plan.ld, tuple(t.shape),
                              "contiguous" if t.is_contiguous() else "strided"))


def execute(plan: Plan, x, mu, sigma, snr, width_idx, ws, stream=None, noise_mode: int = 0):
    """Run ``spd_execute`` on torch CUDA tensors (x: float32 [ndm, ld]; snr float32;
    width_idx int16/uint16; mu, sigma float32 [ndm], or [ndm, n_widths] with noise_mode 1)."""
    _need("execute", plan, x=x, snr=snr, width_idx=width_idx)
    spd_execute(plan, _ptr(x), _ptr(mu), _ptr(sigma), _ptr(snr), _ptr(width_idx), _ptr(ws),
                ws.numel() * ws.element_size(), _stream(stream), noise_mode=noise_mode)


def candidates(plan: Plan, snr, width_idx, threshold: float, peak_radius: int, out, count, ws,
               use_tile_max: bool = False, stream=None):
    """Run ``spd_candidates``; ``out`` is a uint8 CUDA tensor of cap*24 bytes, ``count`` int64[1]."""
    _need("candidates", plan, snr=snr, width_idx=width_idx)
    cap = 0 if out is None else out.numel() * out.element_size() // CANDIDATE_DTYPE.itemsize
    spd_candidates(plan, _ptr(snr), _ptr(width_idx), threshold, peak_radius, _ptr(out), cap,
                   _ptr(count), _ptr(ws), ws.numel() * ws.element_size(), int(bool(use_tile_max)),
                   _stream(stream))


def search(plan: Plan, x, mu, sigma, snr, width_idx, threshold: float, peak_radius: int, out, count,
           ws, stream=None, noise_mode: int = 0):
    """Run ``spd_search`` (search + candidates) on torch CUDA tensors."""
    _need("search", plan, x=x, snr=snr, width_idx=width_idx)
    cap = 0 if out is None else out.numel() * out.element_size() // CANDIDATE_DTYPE.itemsize
    spd_search(plan, _ptr(x), _ptr(mu), _ptr(sigma), _ptr(snr), _ptr(width_idx), threshold,
               peak_radius, _ptr(out), cap, _ptr(count), _ptr(ws), ws.numel() * ws.element_size(),
               _stream(stream), noise_mode=noise_mode)


def noise_stats(plan: Plan, x, mu_out, sigma_out, ws, outlier_sigma: float = 2.0,
                max_passes: int = 10, stream=None):
    """Run ``spd_noise_stats``: fills float32 [ndm, n_widths] mu_out, sigma_out (the
    table of ``execute(..., noise_mode=1)``)."""
    _need("noise_stats", plan, x=x)
    spd_noise_stats(plan, _ptr(x), outlier_sigma, max_passes, _ptr(mu_out), _ptr(sigma_out),
                    _ptr(ws), ws.numel() * ws.element_size(), _stream(stream))


def batch_execute(batch: Batch, xs, ys, widxs, mus, sigmas, ws, readys=None, stream=None):
    """Run ``spd_batch_execute`` on per-range torch CUDA tensors."""
    spd_batch_execute(batch, [_ptr(x) for x in xs], [_ptr(y) for y in ys], [_ptr(w) for w in widxs],
                      [_ptr(m) for m in mus], [_ptr(s) for s in sigmas], _ptr(ws),
                      ws.numel() * ws.element_size(), _stream(stream),
                      readys=None if readys is None else [_ptr(r) for r in readys])


# ----------------------------------------------------------------------------- proposal network
def spd_net_param_count() -> int:
    return int(load_library().spd_net_param_count())


def net_decimate(x, mu, sigma, out, dtype: int = SPD_F32, stream=None):
    """x: [ndm, ld] torch tensor of the dtype's storage; out: float32 [ndm, nt // 16] (nt = x's width)."""
    ndm, ld = x.shape
    nt = out.shape[1] * 16
    _check(load_library().spd_net_decimate(_ptr(x), int(dtype), ndm, nt, ld, _ptr(mu), _ptr(sigma), _ptr(out),
                                           _stream(stream) or None), "spd_net_decimate")


def net_forward(params, blocks, logits, stream=None):
    _check(load_library().spd_net_forward(_ptr(params), _ptr(blocks), blocks.shape[0], _ptr(logits),
                                          _stream(stream) or None), "spd_net_forward")


def net_gradient(params, blocks, labels, grad_sum, loss_sum, stream=None):
    _check(load_library().spd_net_gradient(_ptr(params), _ptr(blocks), _ptr(labels), blocks.shape[0],
                                           _ptr(grad_sum), _ptr(loss_sum), _stream(stream) or None),
           "spd_net_gradient")


def spd_net_gradient_workspace_size() -> int:
    return int(load_library().spd_net_gradient_workspace_size())


def net_gradient_ordered(params, blocks, labels, grad_sum, loss_sum, ws, stream=None):
    """net_gradient with a deterministic sum over the CTAs (``ws``: uint8 CUDA
    tensor of spd_net_gradient_workspace_size() bytes)."""
    _check(load_library().spd_net_gradient_ordered(_ptr(params), _ptr(blocks), _ptr(labels), blocks.shape[0],
                                                   _ptr(grad_sum), _ptr(loss_sum), _ptr(ws),
                                                   ws.numel() * ws.element_size(), _stream(stream) or None),
           "spd_net_gradient_ordered")


def net_adam(params, m, v, grad_sum, n_blocks: int, lr: float, step: int, stream=None):
    _check(load_library().spd_net_adam(_ptr(params), _ptr(m), _ptr(v), _ptr(grad_sum), int(n_blocks),
                                       float(lr), int(step), _stream(stream) or None), "spd_net_adam")


def net_select(logits, threshold: float, out_list, count, stream=None):
    """Ids of the logits above ``threshold`` into the int64 tensor ``out_list`` (in no
    fixed order); their number into the int64[1] tensor ``count``."""
    _check(load_library().spd_net_select(_ptr(logits), logits.numel(), float(threshold), _ptr(out_list),
                                         out_list.numel(), _ptr(count), _stream(stream) or None),
           "spd_net_select")


def net_gather(x, block_ids, n: int, block: int, left: int, width: int, out, dtype: int = SPD_F32, nt=None,
               stream=None):
    """Rows of ``out`` ([n, ld_out] of the dtype's storage) = samples
    b * block - left .. + width - 1 of the rows of ``x`` ([ndm, ld]) named by the
    first ``n`` ids r * ceil(nt / block) + b of ``block_ids``; -inf elsewhere."""
    ndm, ld = x.shape
    nt = ld if nt is None else int(nt)
    if n > block_ids.numel() or out.shape[0] < n:
        raise SpdError(5, "net_gather: %d ids for a list of %d and %d output rows" % (n, block_ids.numel(),
                                                                                      out.shape[0]))
    _check(load_library().spd_net_gather(_ptr(x), int(dtype), ndm, nt, ld, _ptr(block_ids), int(n), int(block),
                                         int(left), int(width), _ptr(out), out.shape[1],
                                         _stream(stream) or None), "spd_net_gather")


def propose_search(prop: Proposal, params, x, mu, sigma, out, count, ws, logit_threshold: float = 0.0,
                   threshold: float = 6.0, noise_mode: int = 0, stream=None) -> int:
    """Run ``spd_propose_search`` on torch CUDA tensors (``x`` [ndm, ld] of the
    proposal's dtype; ``out`` uint8 of cap * 24 bytes; ``count`` int64[1]).
    Returns the number of flagged blocks."""
    if not x.is_contiguous() or x.numel() < prop.ndm * prop.ld:
        raise SpdError(5, "propose_search: x must be contiguous with ndm * ld elements")
    cap = 0 if out is None else out.numel() * out.element_size() // CANDIDATE_DTYPE.itemsize
    return spd_propose_search(prop, _ptr(params), _ptr(x), _ptr(mu), _ptr(sigma), logit_threshold, threshold,
                              _ptr(out), cap, _ptr(count), _ptr(ws), ws.numel() * ws.element_size(),
                              _stream(stream), noise_mode=noise_mode)


def search_blocks(prop: Proposal, x, mu, sigma, ids, out, count, ws, threshold: float = 6.0, noise_mode: int = 0,
                  stream=None):
    """Run ``spd_search_blocks`` on torch CUDA tensors (``ids`` int64, increasing)."""
    if not x.is_contiguous() or x.numel() < prop.ndm * prop.ld:
        raise SpdError(5, "search_blocks: x must be contiguous with ndm * ld elements")
    cap = 0 if out is None else out.numel() * out.element_size() // CANDIDATE_DTYPE.itemsize
    spd_search_blocks(prop, _ptr(x), _ptr(mu), _ptr(sigma), _ptr(ids), ids.numel(), threshold, _ptr(out), cap,
                      _ptr(count), _ptr(ws), ws.numel() * ws.element_size(), _stream(stream), noise_mode=noise_mode)


def records(out_tensor, count: int):
    """Host copy of the first ``count`` candidate records as a numpy structured array."""
    raw = out_tensor[: count * CANDIDATE_DTYPE.itemsize].cpu().numpy()
    return raw.view(CANDIDATE_DTYPE)
