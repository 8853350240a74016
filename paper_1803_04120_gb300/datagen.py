"""Seeded synthetic inputs for the self-join workloads.

This module only draws random numbers; it holds none of the join's
arithmetic, so both the CUDA path and the CPU oracle may be fed from it.

Every stream is counter based: value k of stream (seed, sub) is the
splitmix64 output for state ``seed * G + (sub << 40) + (k + 1) * G`` with
``G = 0x9E3779B97F4A7C15`` (the splitmix64 increment), so the same numbers
come out on any machine and any chunking.  A uniform double in [0, 1) is
``(z >> 11) * 2^-53``.

Every derived value (Gaussian deviates, log-uniform draws, the epsilon of a
target neighbour count) is computed with IEEE-exact operations only (+, -, *,
/, sqrt, frexp, ldexp) through the series in ``_ln``, ``_exp`` and ``_root``,
never with the platform's libm: the same bits come out on x86-64 and on
AArch64, so expected values stored by the oracle on one machine hold on the
other.

Workloads (the paper's synthetic datasets, Section VI-A: coordinates i.i.d.
uniform in [0, 100]^n, FP64):
  * ``uniform(n, d, seed)`` -- the Syn- datasets.
  * ``eps_for_neighbors(n, d, k)`` -- the epsilon at which a ball holds k
    points on average at the uniform density n / 100^d (boundary effects
    lower the realised mean).
  * ``clustered(n, d, seed)`` -- skewed density: 90 % of the points from
    1,000 isotropic Gaussian clusters (centres uniform in [0, 100]^d, sigma
    log-uniform in [0.1, 5], cluster chosen uniformly), 10 % uniform;
    ``side`` widens the domain of the centres and the background.
  * ``serving_requests(count, seed)`` -- a request stream of self-joins of
    uneven size and dimension with Poisson arrivals.
"""
from __future__ import annotations

import numpy as np

_G = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_CHUNK = 1 << 22


def _splitmix(state: np.ndarray) -> np.ndarray:
    z = state.copy()
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def raw64(seed: int, sub: int, count: int, start: int = 0) -> np.ndarray:
    """``count`` raw 64-bit values of stream (seed, sub) from index ``start``."""
    out = np.empty(count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        base = (np.uint64(seed & (2**64 - 1)) * _G + np.uint64((sub << 40) & (2**64 - 1)))
        for c0 in range(0, count, _CHUNK):
            c1 = min(count, c0 + _CHUNK)
            k = np.arange(start + c0 + 1, start + c1 + 1, dtype=np.uint64)
            out[c0:c1] = _splitmix(base + k * _G)
    return out


def unit(seed: int, sub: int, count: int, start: int = 0) -> np.ndarray:
    """``count`` uniform doubles in [0, 1)."""
    z = raw64(seed, sub, count, start)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform(n: int, d: int, seed: int, lo: float = 0.0, hi: float = 100.0) -> np.ndarray:
    """(n, d) row-major FP64 points uniform in [lo, hi)^d."""
    u = unit(seed, 0, n * d)
    if lo == 0.0:
        return (u * hi).reshape(n, d)
    return (lo + u * (hi - lo)).reshape(n, d)


_LN2 = 0.6931471805599453          # ln 2 rounded to double
_SQRT_HALF = 0.7071067811865476    # sqrt(1/2) rounded to double
_PI = 3.141592653589793            # pi rounded to double


def _ln(x) -> np.ndarray:
    """Natural logarithm of positive finite doubles from IEEE-exact steps:
    x = m 2^e with m in [sqrt(1/2), sqrt(2)), ln m = 2 atanh(t) with
    t = (m - 1) / (m + 1), |t| <= 0.1716, summed as the odd series to the
    t^25 term (remainder below 1e-20)."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)
    small = m < _SQRT_HALF
    m = np.where(small, m * 2.0, m)
    e = np.where(small, e - 1, e).astype(np.float64)
    t = (m - 1.0) / (m + 1.0)
    t2 = t * t
    acc = np.full_like(t, 1.0 / 25.0)
    for k in range(11, -1, -1):
        acc = acc * t2 + 1.0 / (2 * k + 1)
    return 2.0 * t * acc + e * _LN2


def _exp(x) -> np.ndarray:
    """exp of doubles in about [-700, 700] from IEEE-exact steps: x = k ln 2
    + r with |r| <= ln 2, exp(r) as its Taylor series to the r^24 term
    (remainder below 1e-24), then scaled by 2^k exactly."""
    x = np.asarray(x, dtype=np.float64)
    k = np.floor(x / _LN2 + 0.5)
    r = x - k * _LN2
    acc = np.ones_like(r)
    for n in range(24, 0, -1):
        acc = acc * (r / float(n)) + 1.0
    return np.ldexp(acc, k.astype(np.int64))


def _root(x: float, d: int) -> float:
    """x^(1/d) for x > 0: a start from _exp(_ln(x) / d), then Newton steps
    y <- y - (y^d - x) / (d y^(d-1)) in plain arithmetic."""
    y = float(_exp(_ln(x) / d))
    for _ in range(4):
        yd1 = 1.0
        for _ in range(d - 1):
            yd1 *= y
        y = y - (yd1 * y - x) / (d * yd1)
    return y


def normals(seed: int, sub: int, count: int) -> np.ndarray:
    """``count`` standard normal deviates by Marsaglia's polar method on the
    uniform streams (seed, sub) and (seed, sub + 1): pairs (v1, v2) uniform
    in [-1, 1)^2 are kept when 0 < s = v1^2 + v2^2 < 1 and give
    v1 f, v2 f with f = sqrt(-2 ln s / s)."""
    need = (count + 1) // 2
    parts, got, start = [], 0, 0
    while got < need:
        cnt = int((need - got) * 1.3) + 1024
        v1 = 2.0 * unit(seed, sub, cnt, start) - 1.0
        v2 = 2.0 * unit(seed, sub + 1, cnt, start) - 1.0
        s = v1 * v1 + v2 * v2
        ok = (s > 0.0) & (s < 1.0)
        v1, v2, s = v1[ok], v2[ok], s[ok]
        f = np.sqrt(-2.0 * _ln(s) / s)
        parts.append(np.stack([v1 * f, v2 * f], axis=1).reshape(-1))
        got += int(ok.sum())
        start += cnt
    return np.concatenate(parts)[:count]


def ball_volume(d: int) -> float:
    """Volume of the unit ball in d dimensions, pi^(d/2) / Gamma(d/2 + 1):
    pi^k / k! for d = 2k, 2^(k+1) pi^k / (2k+1)!! for d = 2k + 1."""
    v = 1.0
    if d % 2 == 0:
        for i in range(1, d // 2 + 1):
            v = v * _PI / i
    else:
        v = 2.0
        for i in range(1, d // 2 + 1):
            v = v * 2.0 * _PI / (2 * i + 1)
    return v


def eps_for_neighbors(n: int, d: int, k: float, side: float = 100.0) -> float:
    """epsilon with ball volume x density = k (self excluded)."""
    sd = 1.0
    for _ in range(d):
        sd *= side
    rho = n / sd
    return _root(k / (ball_volume(d) * rho), d)


_LN50 = 3.912023005428146          # ln 50 rounded to double


def clustered(n: int, d: int, seed: int, clusters: int = 1000,
              frac_clustered: float = 0.9, side: float = 100.0) -> np.ndarray:
    """Skewed-density points (see module docstring), FP64, not clipped.
    ``side`` scales the domain of the centres and of the background
    (the cluster widths stay in [0.1, 5])."""
    centres = unit(seed, 1, clusters * d).reshape(clusters, d) * side
    lu = unit(seed, 2, clusters)
    sigma = 0.1 * _exp(lu * _LN50)          # log-uniform in [0.1, 5)
    n_cl = int(round(n * frac_clustered))
    which = np.minimum((unit(seed, 3, n_cl) * clusters).astype(np.int64), clusters - 1)
    g = normals(seed, 4, n_cl * d)
    pts_cl = centres[which] + g.reshape(n_cl, d) * sigma[which][:, None]
    pts_bg = unit(seed, 6, (n - n_cl) * d).reshape(n - n_cl, d) * side
    pts = np.concatenate([pts_cl, pts_bg], axis=0)
    perm = np.argsort(raw64(seed, 7, n), kind="stable")
    return np.ascontiguousarray(pts[perm])


def serving_requests(count: int, seed: int, rate_hz: float = 1000.0,
                     n_lo: float = 1e3, n_hi: float = 1e6):
    """List of dicts {arrival_s, n, d, k, eps, seed} for a stream of
    self-join requests: Poisson arrivals at ``rate_hz``, n log-uniform in
    [n_lo, n_hi], d uniform in {2..6}, k uniform in [8, 128] nominal
    neighbours, points uniform in [0, 100]^d drawn from the request's seed."""
    u = unit(seed, 10, 4 * count).reshape(count, 4)
    gaps = -_ln(1.0 - u[:, 0]) / rate_hz
    arrivals = np.cumsum(gaps)
    l_lo, l_hi = float(_ln(n_lo)), float(_ln(n_hi))
    ns = _exp(l_lo + u[:, 1] * (l_hi - l_lo)).astype(np.int64)
    ds = 2 + np.minimum((u[:, 2] * 5).astype(np.int64), 4)
    ks = 8.0 + u[:, 3] * 120.0
    out = []
    for r in range(count):
        n, d = int(ns[r]), int(ds[r])
        out.append(dict(arrival_s=float(arrivals[r]), n=n, d=d, k=float(ks[r]),
                        eps=eps_for_neighbors(n, d, float(ks[r])),
                        seed=int(seed * 1000003 + r)))
    return out


# The five workloads, by name.
CONFIG1 = dict(name="uniform-2d-20k", n=20000, d=2, seed=1, eps=2.0)


def config2(d: int) -> dict:
    """2,000,000 uniform points in [0,100]^d, 64 mean neighbours."""
    return dict(name=f"uniform-{d}d-2M", n=2_000_000, d=d, seed=2 + d,
                eps=eps_for_neighbors(2_000_000, d, 64))


def config3(d: int) -> dict:
    """10,000,000 uniform points in [0,100]^d, 128 mean neighbours."""
    return dict(name=f"uniform-{d}d-10M", n=10_000_000, d=d, seed=20 + d,
                eps=eps_for_neighbors(10_000_000, d, 128))


def config4(d: int) -> dict:
    """5,000,000 clustered points, eps = 0.5."""
    return dict(name=f"clustered-{d}d-5M", n=5_000_000, d=d, seed=40 + d, eps=0.5)


def wide_clustered(d: int) -> dict:
    """2,000,000 clustered points spread over [0, 1e6]^d (20,000 clusters of
    about 90 points), eps = 0.5: about 2e6 cells per dimension, where the
    FP32 records relative to g_min lose the precision the filter needs."""
    return dict(name=f"wide-clustered-{d}d-2M", n=2_000_000, d=d, seed=60 + d, eps=0.5,
                clusters=20000, side=1e6)


def make_points(cfg: dict) -> np.ndarray:
    if cfg["name"].startswith("wide-clustered"):
        return clustered(cfg["n"], cfg["d"], cfg["seed"], clusters=cfg["clusters"],
                         side=cfg["side"])
    if cfg["name"].startswith("clustered"):
        return clustered(cfg["n"], cfg["d"], cfg["seed"])
    return uniform(cfg["n"], cfg["d"], cfg["seed"])
