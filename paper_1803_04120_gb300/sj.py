"""Python binding of the C ABI in ``include/sj.h`` (ctypes, marshalling only).

Every function here converts arguments and calls the function of the same
name in ``libsj.so``; all of the join runs in the library's CUDA kernels.
There is no fallback: if the library cannot be built or loaded, or no CUDA
device is present, the calls raise.

Host arrays are numpy arrays; device arrays are torch CUDA tensors (torch is
used only to own device memory and streams).  Pairs come back as an
``(count, 2)`` uint32 array of (i, j) point ids.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

SJ_OK, SJ_PENDING = 0, 1
SJ_EINVAL, SJ_ENOMEM, SJ_ERANGE, SJ_ECUDA = -1, -2, -3, -4
SJ_ETIMEOUT, SJ_EBUSY, SJ_EOVERFLOW, SJ_ENOTFOUND = -5, -6, -7, -8
SJ_PREC_FP64, SJ_PREC_FP32_RECHECK = 0, 1
SJ_LOOKUP_AUTO, SJ_LOOKUP_DENSE, SJ_LOOKUP_SEARCH, SJ_LOOKUP_COORDS = 0, 1, 2, 3
SJ_FRAME_AUTO, SJ_FRAME_GRID, SJ_FRAME_CELL = -1, 0, 1

# symbols the header declares (checked by the CPU test suite)
ABI_FUNCTIONS = (
    "sj_config_default", "sj_create", "sj_destroy", "sj_last_error", "sj_status_str",
    "sj_build_index", "sj_index_free", "sj_index_info", "sj_index_export",
    "sj_selfjoin", "sj_selfjoin_index", "sj_selfjoin_device", "sj_selfjoin_index_device",
    "sj_selfjoin_count", "sj_selfjoin_stream", "sj_result_count", "sj_result_pairs",
    "sj_result_free", "sj_last_stats", "sj_profile_read", "sj_submit", "sj_poll",
    "sj_result_times", "sj_fp32_margin", "sj_selfjoin_noalloc", "sj_selfjoin_multi",
    "sj_serve_stats", "sj_selfjoin_shard_device", "sj_shard_bounds", "sj_shard_bounds_cost",
    "sj_selfjoin_bruteforce_device", "sj_join2_device", "sj_fp32_margin_frame",
    "sj_fp32_margin_diff", "sj_fp32_margin_hd", "sj_fp32_fma_rate", "sj_fp64_fma_rate",
    "sj_tune_reset",
)


class SJError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{status_name(status)}: {message}")
        self.status = status


class sj_config(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int32), ("unicomp", ctypes.c_int32),
                ("out_cap_bytes", ctypes.c_uint64), ("min_batches", ctypes.c_int32),
                ("sorted", ctypes.c_int32), ("autotune", ctypes.c_int32),
                ("device", ctypes.c_int32), ("lookup", ctypes.c_int32),
                ("profile", ctypes.c_int32), ("max_inflight", ctypes.c_int32),
                ("serve_mem_bytes", ctypes.c_uint64), ("grab", ctypes.c_int32),
                ("nbuf", ctypes.c_int32), ("staging", ctypes.c_int32), ("wpb", ctypes.c_int32),
                ("slots", ctypes.c_int32), ("frame", ctypes.c_int32),
                ("wait_ms", ctypes.c_int32), ("test_stall", ctypes.c_int32)]


class sj_index_desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("d", ctypes.c_int32), ("dense", ctypes.c_int32),
                ("eps", ctypes.c_double), ("cell_width", ctypes.c_double),
                ("n_cells", ctypes.c_uint64), ("grid_cells", ctypes.c_uint64),
                ("gmin", ctypes.c_double * 8), ("gmax", ctypes.c_double * 8),
                ("ng", ctypes.c_int64 * 8), ("device_bytes", ctypes.c_uint64),
                ("fp32", ctypes.c_int32), ("frame", ctypes.c_int32),
                ("grid_d", ctypes.c_int32), ("grid_dim", ctypes.c_int32 * 8)]


class sj_stats(ctypes.Structure):
    _fields_ = [("pairs", ctypes.c_uint64), ("evaluations", ctypes.c_uint64),
                ("rechecks", ctypes.c_uint64), ("n_cells", ctypes.c_uint64),
                ("batches", ctypes.c_uint32), ("retries", ctypes.c_uint32),
                ("estimate", ctypes.c_uint64), ("ms_index", ctypes.c_double),
                ("ms_join", ctypes.c_double), ("ms_total", ctypes.c_double),
                ("kernel_launches", ctypes.c_uint64), ("grab", ctypes.c_int32),
                ("nbuf", ctypes.c_int32), ("wpb", ctypes.c_int32), ("tuned", ctypes.c_int32),
                ("staging", ctypes.c_int32), ("frame", ctypes.c_int32)]


class sj_job(ctypes.Structure):
    _fields_ = [("pts", ctypes.c_void_p), ("n", ctypes.c_uint64), ("d", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("eps", ctypes.c_double)]


class sj_serve_info(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("waves", ctypes.c_uint64), ("max_wave", ctypes.c_uint64),
                ("overflow_reruns", ctypes.c_uint64), ("standalone", ctypes.c_uint64),
                ("graph_launches", ctypes.c_uint64), ("queued", ctypes.c_uint64),
                ("mem_in_use", ctypes.c_uint64), ("inflight", ctypes.c_int32),
                ("lanes", ctypes.c_int32), ("max_concurrent_waves", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("ms_bounds", ctypes.c_double),
                ("ms_graph", ctypes.c_double), ("ms_output", ctypes.c_double),
                ("tuned_waves", ctypes.c_uint64), ("ms_tune", ctypes.c_double)]


CHUNK_CB = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.POINTER(ctypes.c_uint32), ctypes.c_uint64,
                            ctypes.c_void_p)

_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load(build: bool = True):
    """Load libsj.so (building it first when out of date)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build() if build else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path}")
        lib = ctypes.CDLL(path)
        P, u64, i32, f64 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_double
        PP = ctypes.POINTER(ctypes.c_void_p)
        sig = {
            "sj_config_default": (None, [ctypes.POINTER(sj_config)]),
            "sj_tune_reset": (None, []),
            "sj_create": (i32, [ctypes.POINTER(sj_config), PP]),
            "sj_destroy": (None, [P]),
            "sj_last_error": (ctypes.c_char_p, [P]),
            "sj_status_str": (ctypes.c_char_p, [i32]),
            "sj_build_index": (i32, [P, P, u64, i32, f64, PP]),
            "sj_index_free": (None, [P]),
            "sj_index_info": (i32, [P, ctypes.POINTER(sj_index_desc)]),
            "sj_index_export": (i32, [P, P, P, P, P]),
            "sj_selfjoin": (i32, [P, P, u64, i32, f64, PP]),
            "sj_selfjoin_index": (i32, [P, P, PP]),
            "sj_selfjoin_device": (i32, [P, P, u64, i32, f64, P, u64,
                                         ctypes.POINTER(ctypes.c_uint64), P]),
            "sj_selfjoin_index_device": (i32, [P, P, P, u64, ctypes.POINTER(ctypes.c_uint64), P]),
            "sj_selfjoin_count": (i32, [P, P, u64, i32, f64, ctypes.POINTER(ctypes.c_uint64)]),
            "sj_selfjoin_stream": (i32, [P, P, u64, i32, f64, CHUNK_CB, P]),
            "sj_result_count": (u64, [P]),
            "sj_result_pairs": (P, [P]),
            "sj_result_free": (None, [P]),
            "sj_last_stats": (i32, [P, ctypes.POINTER(sj_stats)]),
            "sj_profile_read": (i32, [P, ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_uint64)]),
            "sj_submit": (i32, [P, P, u64, i32, f64, ctypes.POINTER(ctypes.c_uint64)]),
            "sj_poll": (i32, [P, u64, i32, PP]),
            "sj_result_times": (i32, [P, ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_double)]),
            "sj_fp32_margin": (i32, [i32, f64, P, P, ctypes.POINTER(ctypes.c_float),
                                     ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)]),
            "sj_fp32_fma_rate": (i32, [i32, i32, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double)]),
            "sj_fp64_fma_rate": (i32, [i32, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double)]),
            "sj_fp32_margin_diff": (i32, [i32, f64, P, P, ctypes.POINTER(ctypes.c_float),
                                          ctypes.POINTER(ctypes.c_float)]),
            "sj_fp32_margin_hd": (i32, [i32, f64, P, P, P, ctypes.POINTER(ctypes.c_float),
                                        ctypes.POINTER(ctypes.c_float), P]),
            "sj_fp32_margin_frame": (i32, [i32, f64, P, P, i32, ctypes.POINTER(ctypes.c_float),
                                           ctypes.POINTER(ctypes.c_float),
                                           ctypes.POINTER(ctypes.c_float)]),
            "sj_selfjoin_noalloc": (i32, [P, u64, i32, f64, P, u64, ctypes.POINTER(ctypes.c_uint64),
                                          P, ctypes.c_char_p, ctypes.c_size_t]),
            "sj_selfjoin_multi": (i32, [P, ctypes.POINTER(sj_job), u64, PP, ctypes.POINTER(ctypes.c_int)]),
            "sj_serve_stats": (i32, [P, ctypes.POINTER(sj_serve_info)]),
            "sj_selfjoin_shard_device": (i32, [P, P, u64, i32, f64, i32, i32, P, u64,
                                               ctypes.POINTER(ctypes.c_uint64), P]),
            "sj_shard_bounds_cost": (i32, [P, P, u64, i32, i32, ctypes.POINTER(ctypes.c_uint64),
                                           ctypes.POINTER(ctypes.c_uint64)]),
            "sj_shard_bounds": (i32, [P, u64, i32, i32, ctypes.POINTER(ctypes.c_uint64),
                                      ctypes.POINTER(ctypes.c_uint64)]),
            "sj_selfjoin_bruteforce_device": (i32, [P, P, u64, i32, f64, P, u64,
                                                    ctypes.POINTER(ctypes.c_uint64), P]),
            "sj_join2_device": (i32, [P, P, u64, P, u64, i32, f64, P, u64,
                                      ctypes.POINTER(ctypes.c_uint64), P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def status_name(st: int) -> str:
    try:
        return load().sj_status_str(st).decode()
    except Exception:  # pragma: no cover
        return str(st)


# ------------------------------------------------------------------ marshalling

def _host_points(points) -> np.ndarray:
    a = np.ascontiguousarray(points, dtype=np.float64)
    if a.ndim != 2:
        raise ValueError("points must be (n, d)")
    return a


def _points_ptr(points):
    """(pointer, n, d, keepalive) for a numpy array or a torch tensor."""
    if hasattr(points, "data_ptr") and hasattr(points, "is_cuda"):
        t = points
        if t.dtype.__repr__() != "torch.float64" or t.dim() != 2 or not t.is_contiguous():
            raise ValueError("device points must be a contiguous (n, d) float64 tensor")
        return ctypes.c_void_p(t.data_ptr()), t.shape[0], t.shape[1], t
    a = _host_points(points)
    return ctypes.c_void_p(a.ctypes.data), a.shape[0], a.shape[1], a


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _result_to_numpy(lib, r) -> np.ndarray:
    n = lib.sj_result_count(r)
    p = lib.sj_result_pairs(r)
    out = np.empty((n, 2), dtype=np.uint32)
    if n:
        ctypes.memmove(out.ctypes.data, p, n * 8)
    return out


class Context:
    """A library context (one CUDA device)."""

    def __init__(self, prec: int = SJ_PREC_FP32_RECHECK, unicomp: bool = True,
                 out_cap_bytes: int = 2 << 30, min_batches: int = 3, sorted: bool = False,
                 device: int = 0, lookup: int = SJ_LOOKUP_AUTO, profile: bool = False,
                 max_inflight: int = 64, serve_mem_bytes: int = 8 << 30, autotune: bool = True,
                 grab: int = -1, nbuf: int = -1, staging: int = -1, wpb: int = -1,
                 slots: int = -1, frame: int = SJ_FRAME_AUTO, wait_ms: int = 0,
                 test_stall: bool = False):
        lib = load()
        cfg = sj_config()
        lib.sj_config_default(ctypes.byref(cfg))
        cfg.prec, cfg.unicomp = prec, int(bool(unicomp))
        cfg.out_cap_bytes, cfg.min_batches, cfg.sorted = out_cap_bytes, min_batches, int(sorted)
        cfg.device, cfg.lookup, cfg.profile = device, lookup, int(profile)
        cfg.max_inflight, cfg.serve_mem_bytes, cfg.autotune = max_inflight, serve_mem_bytes, int(autotune)
        cfg.grab, cfg.nbuf, cfg.staging, cfg.wpb, cfg.slots = grab, nbuf, staging, wpb, slots
        cfg.frame, cfg.wait_ms, cfg.test_stall = frame, int(wait_ms), int(bool(test_stall))
        h = ctypes.c_void_p()
        st = lib.sj_create(ctypes.byref(cfg), ctypes.byref(h))
        if st != SJ_OK:
            raise SJError(st, "sj_create failed")
        self._lib, self._h, self.config = lib, h, cfg

    # -- plumbing
    def close(self):
        if getattr(self, "_h", None):
            self._lib.sj_destroy(self._h)
            self._h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, st: int, what: str):
        if st != SJ_OK:
            raise SJError(st, f"{what}: {self._lib.sj_last_error(self._h).decode()}")

    # -- joins
    def sj_selfjoin(self, points, eps: float) -> np.ndarray:
        """All pairs within eps, host result, as an (count, 2) uint32 array."""
        p, n, d, keep = _points_ptr(points)
        r = ctypes.c_void_p()
        self._check(self._lib.sj_selfjoin(self._h, p, n, d, float(eps), ctypes.byref(r)), "sj_selfjoin")
        try:
            return _result_to_numpy(self._lib, r)
        finally:
            self._lib.sj_result_free(r)

    def sj_selfjoin_raw(self, points, eps: float):
        """Like sj_selfjoin but returns the library's result handle (caller
        frees it with sj_result_free); avoids the copy into numpy."""
        p, n, d, keep = _points_ptr(points)
        r = ctypes.c_void_p()
        self._check(self._lib.sj_selfjoin(self._h, p, n, d, float(eps), ctypes.byref(r)), "sj_selfjoin")
        return r

    def sj_result_count(self, r) -> int:
        return int(self._lib.sj_result_count(r))

    def sj_result_free(self, r):
        self._lib.sj_result_free(r)

    def sj_selfjoin_device(self, points, eps: float, out, stream=None, raise_overflow=True) -> int:
        """Join into a device uint32 tensor ``out`` of shape (cap, 2); returns
        the pair count (which may exceed cap: then SJEOVERFLOW is raised
        unless raise_overflow is False)."""
        p, n, d, keep = _points_ptr(points)
        cap = 0 if out is None else out.shape[0]
        optr = ctypes.c_void_p(out.data_ptr()) if out is not None and cap else None
        cnt = ctypes.c_uint64(0)
        st = self._lib.sj_selfjoin_device(self._h, p, n, d, float(eps), optr, cap,
                                          ctypes.byref(cnt), _stream_ptr(stream))
        if st == SJ_EOVERFLOW and not raise_overflow:
            return int(cnt.value)
        self._check(st, "sj_selfjoin_device")
        return int(cnt.value)

    def sj_selfjoin_shard_device(self, points, eps: float, rank: int, world: int, out,
                                 stream=None, raise_overflow: bool = True) -> int:
        """Rank `rank` of `world`'s share of the join into a device buffer;
        returns its pair count."""
        p, n, d, keep = _points_ptr(points)
        cap = 0 if out is None else out.shape[0]
        optr = ctypes.c_void_p(out.data_ptr()) if out is not None and cap else None
        cnt = ctypes.c_uint64(0)
        st = self._lib.sj_selfjoin_shard_device(self._h, p, n, d, float(eps), int(rank), int(world),
                                                optr, cap, ctypes.byref(cnt), _stream_ptr(stream))
        if st == SJ_EOVERFLOW and not raise_overflow:
            return int(cnt.value)
        self._check(st, "sj_selfjoin_shard_device")
        return int(cnt.value)

    def sj_join2_device(self, R, S, eps: float, out, stream=None, raise_overflow: bool = True) -> int:
        """Two-set join R ⋈ S into a device buffer of (index in R, index in S)
        pairs; returns the pair count."""
        pr, nr, dr, kr = _points_ptr(R)
        ps, ns, ds, ks = _points_ptr(S)
        if dr != ds:
            raise ValueError("R and S must have the same dimension")
        cap = 0 if out is None else out.shape[0]
        optr = ctypes.c_void_p(out.data_ptr()) if out is not None and cap else None
        cnt = ctypes.c_uint64(0)
        st = self._lib.sj_join2_device(self._h, pr, nr, ps, ns, dr, float(eps), optr, cap,
                                       ctypes.byref(cnt), _stream_ptr(stream))
        if st == SJ_EOVERFLOW and not raise_overflow:
            return int(cnt.value)
        self._check(st, "sj_join2_device")
        return int(cnt.value)

    def sj_selfjoin_bruteforce_device(self, points, eps: float, out, stream=None,
                                      raise_overflow: bool = True) -> int:
        """The index-free O(n^2) comparator into a device buffer."""
        p, n, d, keep = _points_ptr(points)
        cap = 0 if out is None else out.shape[0]
        optr = ctypes.c_void_p(out.data_ptr()) if out is not None and cap else None
        cnt = ctypes.c_uint64(0)
        st = self._lib.sj_selfjoin_bruteforce_device(self._h, p, n, d, float(eps), optr, cap,
                                                     ctypes.byref(cnt), _stream_ptr(stream))
        if st == SJ_EOVERFLOW and not raise_overflow:
            return int(cnt.value)
        self._check(st, "sj_selfjoin_bruteforce_device")
        return int(cnt.value)

    def sj_selfjoin_count(self, points, eps: float) -> int:
        p, n, d, keep = _points_ptr(points)
        cnt = ctypes.c_uint64(0)
        self._check(self._lib.sj_selfjoin_count(self._h, p, n, d, float(eps), ctypes.byref(cnt)),
                    "sj_selfjoin_count")
        return int(cnt.value)

    def sj_selfjoin_stream(self, points, eps: float, callback, copy: bool = True) -> None:
        """callback(pairs: np.ndarray (k, 2) uint32) per batch, or callback(k)
        with the batch's pair count only when copy is False; return True to
        stop."""
        p, n, d, keep = _points_ptr(points)

        def tramp(ptr, k, user):
            if not copy:
                return 1 if callback(int(k)) else 0
            arr = np.ctypeslib.as_array(ptr, shape=(int(k) * 2,)).reshape(-1, 2).copy()
            return 1 if callback(arr) else 0

        cb = CHUNK_CB(tramp)
        self._check(self._lib.sj_selfjoin_stream(self._h, p, n, d, float(eps), cb, None),
                    "sj_selfjoin_stream")

    # -- index
    def sj_build_index(self, points, eps: float) -> "Index":
        p, n, d, keep = _points_ptr(points)
        h = ctypes.c_void_p()
        self._check(self._lib.sj_build_index(self._h, p, n, d, float(eps), ctypes.byref(h)),
                    "sj_build_index")
        return Index(self, h)

    def sj_selfjoin_index(self, index: "Index") -> np.ndarray:
        r = ctypes.c_void_p()
        self._check(self._lib.sj_selfjoin_index(self._h, index._h, ctypes.byref(r)),
                    "sj_selfjoin_index")
        try:
            return _result_to_numpy(self._lib, r)
        finally:
            self._lib.sj_result_free(r)

    def sj_selfjoin_index_device(self, index: "Index", out, stream=None) -> int:
        cap = 0 if out is None else out.shape[0]
        optr = ctypes.c_void_p(out.data_ptr()) if out is not None and cap else None
        cnt = ctypes.c_uint64(0)
        self._check(self._lib.sj_selfjoin_index_device(self._h, index._h, optr, cap,
                                                        ctypes.byref(cnt), _stream_ptr(stream)),
                    "sj_selfjoin_index_device")
        return int(cnt.value)

    # -- serving
    def sj_submit(self, points, eps: float) -> int:
        p, n, d, keep = _points_ptr(points)
        t = ctypes.c_uint64(0)
        self._check(self._lib.sj_submit(self._h, p, n, d, float(eps), ctypes.byref(t)), "sj_submit")
        return int(t.value)

    def sj_poll(self, ticket: int, wait_ms: int = 0, copy: bool = True):
        """None while pending, else (pairs, (t_submit, t_admit, t_done)) where
        pairs is the (count, 2) uint32 array, or only the count when copy is
        False."""
        r = ctypes.c_void_p()
        st = self._lib.sj_poll(self._h, ticket, int(wait_ms), ctypes.byref(r))
        if st == SJ_PENDING:
            return None
        self._check(st, "sj_poll")
        try:
            ts = [ctypes.c_double() for _ in range(3)]
            self._lib.sj_result_times(r, *[ctypes.byref(x) for x in ts])
            pairs = _result_to_numpy(self._lib, r) if copy else int(self._lib.sj_result_count(r))
            return pairs, tuple(x.value for x in ts)
        finally:
            self._lib.sj_result_free(r)

    def sj_selfjoin_multi(self, jobs, raise_errors: bool = True, copy: bool = True):
        """Joins [(points, eps), ...] together; returns a list with one
        (count, 2) uint32 pair array per job, or only its pair count when copy
        is False (None for a failed job when raise_errors is False)."""
        keep = []
        arr = (sj_job * max(1, len(jobs)))()
        for k, (pts, eps) in enumerate(jobs):
            p, n, d, kp = _points_ptr(pts)
            keep.append(kp)
            arr[k].pts, arr[k].n, arr[k].d, arr[k].eps = p, n, d, float(eps)
        outs = (ctypes.c_void_p * max(1, len(jobs)))()
        stat = (ctypes.c_int * max(1, len(jobs)))()
        st = self._lib.sj_selfjoin_multi(self._h, arr, len(jobs), outs, stat)
        res = []
        try:
            for k in range(len(jobs)):
                if not outs[k]:
                    res.append(None)
                elif copy:
                    res.append(_result_to_numpy(self._lib, ctypes.c_void_p(outs[k])))
                else:
                    res.append(int(self._lib.sj_result_count(ctypes.c_void_p(outs[k]))))
        finally:
            for k in range(len(jobs)):
                if outs[k]:
                    self._lib.sj_result_free(ctypes.c_void_p(outs[k]))
        if raise_errors:
            self._check(st, "sj_selfjoin_multi")
        self.last_multi_status = [int(stat[k]) for k in range(len(jobs))]
        return res

    def sj_serve_stats(self) -> dict:
        s = sj_serve_info()
        self._check(self._lib.sj_serve_stats(self._h, ctypes.byref(s)), "sj_serve_stats")
        return {k: getattr(s, k) for k, _ in sj_serve_info._fields_ if k != "reserved"}

    # -- diagnostics
    def sj_last_stats(self) -> dict:
        s = sj_stats()
        self._check(self._lib.sj_last_stats(self._h, ctypes.byref(s)), "sj_last_stats")
        return {k: getattr(s, k) for k, _ in sj_stats._fields_}

    def sj_profile_read(self):
        ms = ctypes.c_double(0)
        n = ctypes.c_uint64(0)
        self._check(self._lib.sj_profile_read(self._h, ctypes.byref(ms), ctypes.byref(n)),
                    "sj_profile_read")
        return ms.value, int(n.value)


class Index:
    """A device-resident grid index (Section IV-B/C)."""

    def __init__(self, ctx: Context, h):
        self._ctx, self._h = ctx, h

    def free(self):
        if self._h:
            self._ctx._lib.sj_index_free(self._h)
            self._h = None

    def __del__(self):  # pragma: no cover
        try:
            self.free()
        except Exception:
            pass

    def sj_index_info(self) -> dict:
        dsc = sj_index_desc()
        st = self._ctx._lib.sj_index_info(self._h, ctypes.byref(dsc))
        if st != SJ_OK:
            raise SJError(st, "sj_index_info")
        g = dsc.grid_d
        return dict(n=dsc.n, d=dsc.d, dense=dsc.dense, eps=dsc.eps, cell_width=dsc.cell_width,
                    n_cells=dsc.n_cells, grid_cells=dsc.grid_cells,
                    gmin=list(dsc.gmin)[:g], gmax=list(dsc.gmax)[:g], ng=list(dsc.ng)[:g],
                    device_bytes=dsc.device_bytes, fp32=dsc.fp32, frame=dsc.frame,
                    grid_d=g, grid_dim=list(dsc.grid_dim)[:g])

    def sj_index_export(self):
        """(B, G, A, M) as numpy arrays (Section IV-C); B is None for cells
        ordered by coordinate tuple (no linear ids)."""
        info = self.sj_index_info()
        nc, n, d = info["n_cells"], info["n"], info["grid_d"]
        mwords = (max(info["ng"]) + 31) // 32
        B = np.empty(nc, np.uint64)
        G = np.empty(nc + 1, np.uint32)
        A = np.empty(n, np.uint32)
        M = np.empty((d, mwords), np.uint32)
        lib = self._ctx._lib
        st = lib.sj_index_export(self._h, B.ctypes.data, G.ctypes.data, A.ctypes.data, M.ctypes.data)
        if st == SJ_ERANGE:
            B = None
            st = lib.sj_index_export(self._h, None, G.ctypes.data, A.ctypes.data, M.ctypes.data)
        if st != SJ_OK:
            raise SJError(st, "sj_index_export")
        return B, G, A, M


def sj_selfjoin_noalloc(points, eps: float, out, stream=None, raise_overflow: bool = True) -> int:
    """Join for callers that cannot allocate: device points (contiguous
    (n, d) float64 CUDA tensor) into the device tensor ``out`` of shape
    (cap, 2), using only the library's fixed static scratch (n <= 65536).
    Returns the pair count."""
    p, n, d, keep = _points_ptr(points)
    lib = load()
    cap = 0 if out is None else out.shape[0]
    optr = ctypes.c_void_p(out.data_ptr()) if out is not None and cap else None
    cnt = ctypes.c_uint64(0)
    msg = ctypes.create_string_buffer(256)
    st = lib.sj_selfjoin_noalloc(p, n, d, float(eps), optr, cap, ctypes.byref(cnt),
                                 _stream_ptr(stream), msg, 256)
    if st == SJ_EOVERFLOW and not raise_overflow:
        return int(cnt.value)
    if st != SJ_OK:
        raise SJError(st, "sj_selfjoin_noalloc: " + msg.value.decode())
    return int(cnt.value)


def sj_fp32_margin(d: int, eps: float, gmin, gmax):
    """(status, w32, lo, hi) of the FP32 filter margin for a grid (host only)."""
    lib = load()
    gmin = np.ascontiguousarray(gmin, dtype=np.float64)
    gmax = np.ascontiguousarray(gmax, dtype=np.float64)
    w, lo, hi = ctypes.c_float(), ctypes.c_float(), ctypes.c_float()
    st = lib.sj_fp32_margin(d, float(eps), gmin.ctypes.data, gmax.ctypes.data,
                            ctypes.byref(w), ctypes.byref(lo), ctypes.byref(hi))
    return st, w.value, lo.value, hi.value


def sj_fp32_margin_frame(d: int, eps: float, gmin, gmax, frame: int):
    """(status, w32, lo, hi) of the FP32 filter margin for records of the
    given frame (SJ_FRAME_GRID or SJ_FRAME_CELL), host only."""
    lib = load()
    gmin = np.ascontiguousarray(gmin, dtype=np.float64)
    gmax = np.ascontiguousarray(gmax, dtype=np.float64)
    w, lo, hi = ctypes.c_float(), ctypes.c_float(), ctypes.c_float()
    st = lib.sj_fp32_margin_frame(d, float(eps), gmin.ctypes.data, gmax.ctypes.data, int(frame),
                                  ctypes.byref(w), ctypes.byref(lo), ctypes.byref(hi))
    return st, w.value, lo.value, hi.value


def sj_fp32_margin_diff(d: int, eps: float, fmin, fmax):
    """(status, lo, hi) of the FP32 margin used for points of more than 8
    dimensions (difference-form sum; host only)."""
    lib = load()
    fmin = np.ascontiguousarray(fmin, dtype=np.float64)
    fmax = np.ascontiguousarray(fmax, dtype=np.float64)
    lo, hi = ctypes.c_float(), ctypes.c_float()
    st = lib.sj_fp32_margin_diff(d, float(eps), fmin.ctypes.data, fmax.ctypes.data,
                                 ctypes.byref(lo), ctypes.byref(hi))
    return st, lo.value, hi.value


def sj_fp32_margin_hd(d: int, eps: float, fmin, fmax, grid):
    """(status, lo, hi, mid) of the expanded-form FP32 margin for points of
    more than 8 dimensions: grid[j] marks the grid dimensions, mid[j] is the
    origin of the others (host only)."""
    lib = load()
    fmin = np.ascontiguousarray(fmin, dtype=np.float64)
    fmax = np.ascontiguousarray(fmax, dtype=np.float64)
    g = np.ascontiguousarray(grid, dtype=np.int32)
    mid = np.zeros(max(d, 1), dtype=np.float32)
    lo, hi = ctypes.c_float(), ctypes.c_float()
    st = lib.sj_fp32_margin_hd(d, float(eps), fmin.ctypes.data, fmax.ctypes.data, g.ctypes.data,
                               ctypes.byref(lo), ctypes.byref(hi), mid.ctypes.data)
    return st, lo.value, hi.value, mid[:d].copy()


def sj_fp32_fma_rate(device: int = 0, packed: bool = True):
    """(TFLOP/s, ms) of FP32 fused multiply-add chains on every SM of the
    device: scalar fma.rn.f32 or packed fma.rn.f32x2 (two FLOPs per lane)."""
    lib = load()
    tf, ms = ctypes.c_double(), ctypes.c_double()
    st = lib.sj_fp32_fma_rate(int(device), int(bool(packed)), ctypes.byref(tf), ctypes.byref(ms))
    if st != SJ_OK:
        raise SJError(st, "sj_fp32_fma_rate failed")
    return tf.value, ms.value


def sj_fp64_fma_rate(device: int = 0):
    """(TFLOP/s, ms) of FP64 fused multiply-add chains on every SM of the
    device (two FLOPs per FMA)."""
    lib = load()
    tf, ms = ctypes.c_double(), ctypes.c_double()
    st = lib.sj_fp64_fma_rate(int(device), ctypes.byref(tf), ctypes.byref(ms))
    if st != SJ_OK:
        raise SJError(st, "sj_fp64_fma_rate failed")
    return tf.value, ms.value


def sj_tune_reset():
    """Forgets every choice of the launch tuners of the process (single joins
    and many-join waves); the next join or wave of each key is tuned again."""
    load().sj_tune_reset()


def sj_shard_bounds(item_block, rank: int, world: int):
    """(lo, hi) work-item range of a shard from host block indices (no device)."""
    lib = load()
    a = np.ascontiguousarray(item_block, dtype=np.uint32)
    lo, hi = ctypes.c_uint64(0), ctypes.c_uint64(0)
    st = lib.sj_shard_bounds(ctypes.c_void_p(a.ctypes.data) if a.size else None, a.size, int(rank),
                             int(world), ctypes.byref(lo), ctypes.byref(hi))
    if st != SJ_OK:
        raise SJError(st, "sj_shard_bounds")
    return int(lo.value), int(hi.value)


def sj_shard_bounds_cost(item_block, item_cost, rank: int, world: int):
    """(lo, hi) work-item range of a shard balanced by per-item costs, from
    host arrays (no device)."""
    lib = load()
    a = np.ascontiguousarray(item_block, dtype=np.uint32)
    c = np.ascontiguousarray(item_cost, dtype=np.uint64)
    if a.shape != c.shape:
        raise ValueError("item_block and item_cost differ in length")
    lo, hi = ctypes.c_uint64(0), ctypes.c_uint64(0)
    st = lib.sj_shard_bounds_cost(ctypes.c_void_p(a.ctypes.data) if a.size else None,
                                  ctypes.c_void_p(c.ctypes.data) if c.size else None, a.size,
                                  int(rank), int(world), ctypes.byref(lo), ctypes.byref(hi))
    if st != SJ_OK:
        raise SJError(st, "sj_shard_bounds_cost")
    return int(lo.value), int(hi.value)


def pairs_to_keys(pairs: np.ndarray) -> np.ndarray:
    """(count, 2) uint32 pairs -> sorted uint64 keys (i << 32) | j."""
    p = np.asarray(pairs, dtype=np.uint32).reshape(-1, 2)
    k = (p[:, 0].astype(np.uint64) << np.uint64(32)) | p[:, 1].astype(np.uint64)
    k.sort()
    return k
