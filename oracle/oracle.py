"""CPU oracle for the Euclidean epsilon self-join -- TEST INFRASTRUCTURE.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  The library in
``paper_1803_04120_gb300`` never imports it, and this module imports nothing
from the library: the two share no code.

The arithmetic lives in ``sj_oracle.c`` (plain C, FP64, built with
``-ffp-contract=off``); this file only compiles it, loads it with ctypes and
marshals numpy arrays.  What it computes (Section III of Gowanlock & Karsin):
every ordered pair (i, j), self-pairs included, whose Euclidean distance is at
most epsilon, decided bit-exactly as ``s <= fl(eps*eps)`` with
``s = sum_j fl(fl(x_i[j] - x_j[j])^2)`` summed left to right.

Pairs are returned as sorted uint64 keys ``i << 32 | j``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sj_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")

# Flags are part of the oracle's definition: no contraction of a*b+c into an
# FMA, no fast-math, IEEE doubles.
CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
          "-pthread", "-std=c11"]

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``sj_oracle.c`` into ``oracle/_build/liboracle.so``."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        u64, i64, i32, f64 = ctypes.c_uint64, ctypes.c_int64, ctypes.c_int, ctypes.c_double
        lib.sj_oracle_eps2.argtypes = [f64]
        lib.sj_oracle_eps2.restype = f64
        lib.sj_oracle_within.argtypes = [P, P, i32, f64]
        lib.sj_oracle_within.restype = i32
        lib.sj_oracle_sqdist.argtypes = [P, P, i32]
        lib.sj_oracle_sqdist.restype = f64
        lib.sj_oracle_mix64.argtypes = [u64]
        lib.sj_oracle_mix64.restype = u64
        lib.sj_oracle_bruteforce.argtypes = [P, u64, i32, f64, P, u64]
        lib.sj_oracle_bruteforce.restype = i64
        lib.sj_oracle_bruteforce2.argtypes = [P, u64, P, u64, i32, f64, P, u64]
        lib.sj_oracle_bruteforce2.restype = i64
        lib.sj_oracle_grid_cells.argtypes = [P, u64, i32, f64, P, P]
        lib.sj_oracle_grid_cells.restype = i32
        lib.sj_oracle_grid_join.argtypes = [P, u64, i32, f64, i32, P, u64]
        lib.sj_oracle_grid_join.restype = i64
        lib.sj_oracle_grid_digest.argtypes = [P, u64, i32, f64, i32, P, P, P]
        lib.sj_oracle_grid_digest.restype = i32
        lib.sj_oracle_grid_neighbors.argtypes = [P, u64, i32, f64, i32, P, u64, P, P, u64]
        lib.sj_oracle_grid_neighbors.restype = i64
        _lib = lib
        return lib


def _pts(points) -> np.ndarray:
    a = np.ascontiguousarray(points, dtype=np.float64)
    if a.ndim != 2:
        raise ValueError("points must be an (n, d) array")
    return a


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def default_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity")
               else (os.cpu_count() or 1))


def eps2(eps: float) -> float:
    """fl(eps * eps)."""
    return _load().sj_oracle_eps2(float(eps))


def within(a, b, eps: float) -> bool:
    """The member predicate of Section III for two points."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    return bool(_load().sj_oracle_within(_ptr(a), _ptr(b), a.shape[0], float(eps)))


def sqdist(a, b) -> float:
    """The squared distance exactly as the predicate forms it."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    return _load().sj_oracle_sqdist(_ptr(a), _ptr(b), a.shape[0])


def mix64(z: int) -> int:
    """splitmix64 finaliser used by the order-independent pair hash."""
    return int(_load().sj_oracle_mix64(ctypes.c_uint64(z & (2**64 - 1))))


def _check(rc: int, what: str) -> int:
    if rc == -1:
        raise ValueError(f"{what}: invalid input")
    if rc == -2:
        raise MemoryError(f"{what}: out of memory")
    if rc < 0:
        raise RuntimeError(f"{what}: error {rc}")
    return rc


def bruteforce(points, eps: float) -> np.ndarray:
    """All members by the O(n^2) definition, as sorted keys i << 32 | j."""
    p = _pts(points)
    n, d = p.shape
    lib = _load()
    cnt = _check(lib.sj_oracle_bruteforce(_ptr(p), n, d, float(eps), None, 0), "bruteforce")
    out = np.empty(cnt, dtype=np.uint64)
    got = lib.sj_oracle_bruteforce(_ptr(p), n, d, float(eps), _ptr(out), cnt)
    assert got == cnt
    return out


def bruteforce2(R, S, eps: float) -> np.ndarray:
    """The two-set join R ⋈ S by its O(|R| |S|) definition, as sorted keys
    i << 32 | j (i indexes R, j indexes S)."""
    r, s = _pts(R), _pts(S)
    if r.shape[1] != s.shape[1]:
        raise ValueError("R and S must have the same dimension")
    lib = _load()
    args = (_ptr(r), r.shape[0], _ptr(s), s.shape[0], r.shape[1], float(eps))
    cnt = _check(lib.sj_oracle_bruteforce2(*args, None, 0), "bruteforce2")
    out = np.empty(cnt, dtype=np.uint64)
    got = lib.sj_oracle_bruteforce2(*args, _ptr(out), cnt)
    assert got == cnt
    return np.sort(out)


def grid_join(points, eps: float, nthreads: int | None = None) -> np.ndarray:
    """All members via the grid search of Algorithm 1, as sorted keys."""
    p = _pts(points)
    n, d = p.shape
    lib = _load()
    t = nthreads or default_threads()
    cnt = _check(lib.sj_oracle_grid_join(_ptr(p), n, d, float(eps), t, None, 0), "grid_join")
    out = np.empty(cnt, dtype=np.uint64)
    got = lib.sj_oracle_grid_join(_ptr(p), n, d, float(eps), t, _ptr(out), cnt)
    assert got == cnt
    return out


def grid_digest(points, eps: float, nthreads: int | None = None,
                with_degree: bool = True):
    """(count, per-point degree or None, hash) of the member set, where
    hash = sum of mix64(i << 32 | j) over members, mod 2^64."""
    p = _pts(points)
    n, d = p.shape
    deg = np.zeros(n, dtype=np.uint32) if with_degree else None
    cnt = ctypes.c_uint64(0)
    h = ctypes.c_uint64(0)
    rc = _load().sj_oracle_grid_digest(_ptr(p), n, d, float(eps), nthreads or default_threads(),
                                       _ptr(deg) if deg is not None else None,
                                       ctypes.byref(cnt), ctypes.byref(h))
    _check(rc, "grid_digest")
    return int(cnt.value), deg, int(h.value)


def grid_neighbors(points, eps: float, queries, nthreads: int | None = None):
    """Neighbour lists of the listed queries: (offsets[nq+1], ids) with
    ids[offsets[k]:offsets[k+1]] the ascending j of members (queries[k], j)."""
    p = _pts(points)
    n, d = p.shape
    q = np.ascontiguousarray(queries, dtype=np.uint32)
    lib = _load()
    t = nthreads or default_threads()
    offs = np.zeros(q.shape[0] + 1, dtype=np.uint64)
    total = _check(lib.sj_oracle_grid_neighbors(_ptr(p), n, d, float(eps), t, _ptr(q), q.shape[0],
                                                _ptr(offs), None, 0), "grid_neighbors")
    ids = np.empty(total, dtype=np.uint32)
    got = lib.sj_oracle_grid_neighbors(_ptr(p), n, d, float(eps), t, _ptr(q), q.shape[0],
                                       _ptr(offs), _ptr(ids), total)
    assert got == total
    return offs, ids


def grid_neighbor_counts(points, eps: float, queries, nthreads: int | None = None):
    """offsets[nq+1] of the neighbour lists of the listed queries (the counts
    only): one grid build and one search pass, nothing copied out."""
    p = _pts(points)
    n, d = p.shape
    q = np.ascontiguousarray(queries, dtype=np.uint32)
    offs = np.zeros(q.shape[0] + 1, dtype=np.uint64)
    _check(_load().sj_oracle_grid_neighbors(_ptr(p), n, d, float(eps), nthreads or default_threads(),
                                            _ptr(q), q.shape[0], _ptr(offs), None, 0),
           "grid_neighbor_counts")
    return offs


def grid_cells(points, eps: float):
    """(|g_j| per dimension, linear cell id of every point) of the grid of
    Section IV-B as the oracle builds it."""
    p = _pts(points)
    n, d = p.shape
    ng = np.zeros(d, dtype=np.int64)
    cells = np.zeros(n, dtype=np.uint64)
    _check(_load().sj_oracle_grid_cells(_ptr(p), n, d, float(eps), _ptr(ng), _ptr(cells)),
           "grid_cells")
    return ng, cells


def pair_hash(keys: np.ndarray) -> int:
    """Order-independent hash of a key array, the same function the digest
    uses: sum of mix64(key) mod 2^64 (vectorised with numpy)."""
    z = np.asarray(keys, dtype=np.uint64).copy()
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xbf58476d1ce4e5b9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94d049bb133111eb)
        z = z ^ (z >> np.uint64(31))
    return int(z.sum(dtype=np.uint64))
