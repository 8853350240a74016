"""Soundness of the FP32 filter margin (CPU only).

The kernel's FP32 evaluation is emulated here bit-exactly with rational
arithmetic (every operation rounded to nearest FP32 on its own, fused
multiply-adds rounded once), and the exact FP64 member test is evaluated the
same way.  For adversarial pairs placed at the threshold, a value at or below
the library's ``lo`` must be a member and a value above ``hi`` must not be.
"""
import math
from fractions import Fraction as F

import numpy as np
import pytest

from paper_1803_04120_gb300 import sj


def rn(x: F, mant: int, emin: int) -> F:
    """Round a rational to the nearest binary float with `mant` significand
    bits and minimum normal exponent `emin` (ties to even, gradual underflow)."""
    if x == 0:
        return F(0)
    s = -1 if x < 0 else 1
    a = abs(x)
    e = math.floor(math.log2(a.numerator) - math.log2(a.denominator))
    # fix the estimate so that 2^e <= a < 2^(e+1)
    while F(2) ** e > a:
        e -= 1
    while F(2) ** (e + 1) <= a:
        e += 1
    e = max(e, emin)
    q = a / F(2) ** (e - mant + 1)
    n, r = divmod(q.numerator, q.denominator)
    rem = F(r, q.denominator)
    if rem > F(1, 2) or (rem == F(1, 2) and n % 2 == 1):
        n += 1
    return s * F(n) * F(2) ** (e - mant + 1)


def r32(x):
    return rn(F(x), 24, -126)


def r64(x):
    return rn(F(x), 53, -1022)


def exact_member(a, b, E2):
    s = F(0)
    for x, y in zip(a, b):
        t = r64(F(x) - F(y))
        s = r64(s + r64(t * t))
    return s <= E2


def cell_of(x, gmin, inv_w, ng):
    q = float(r64(r64(F(x) - F(gmin)) * F(inv_w)))
    return min(max(int(math.floor(q)), 0), ng - 1)


def kernel_s32(p, q, gmin, w32, cells):
    """s32 as the kernel computes it for query p (home cell `cells`) and
    candidate q."""
    d = len(p)
    zp, zq = [], []
    for j in range(d):
        o = r32(r32(F(cells[j]) + F(1, 2)) * F(w32))
        yp = r32(r64(F(p[j]) - F(gmin[j])))
        yq = r32(r64(F(q[j]) - F(gmin[j])))
        zp.append(r32(yp - o))
        zq.append(r32(yq - o))
    pp = F(0)
    qq = F(0)
    for j in range(d):
        pp = r32(zp[j] * zp[j] + pp)
        qq = r32(zq[j] * zq[j] + qq)
    acc = r32(qq + pp)
    for j in range(d):
        acc = r32((-2 * zp[j]) * zq[j] + acc)
    return acc


@pytest.mark.parametrize("d,eps,scale,offset", [
    (2, 0.31915, 100.0, 0.0), (3, 1.96949, 100.0, 0.0), (6, 13.55112, 100.0, 0.0),
    (2, 0.37, 30.0, -1e6), (8, 0.9, 10.0, 5.0), (1, 0.05, 1000.0, 0.0)])
def test_margin_sound_on_threshold_pairs(d, eps, scale, offset):
    rng = np.random.default_rng(int(eps * 1000) + d)
    pts = offset + rng.uniform(0, scale, size=(60, d))
    extra = []
    for p in pts:
        v = rng.normal(size=d)
        v /= np.linalg.norm(v)
        for f in (1.0, 1.0 + 2.0 ** -52, 1.0 - 2.0 ** -52, 1.0 + 3e-7, 1.0 - 3e-7,
                  1.0 + 2e-6, 1.0 - 2e-6):
            extra.append(p + v * eps * f)
    allp = np.concatenate([pts, np.array(extra)])
    gmin = allp.min(axis=0) - eps
    gmax = allp.max(axis=0) + eps
    st, w32, lo, hi = sj.sj_fp32_margin(d, eps, gmin, gmax)
    assert st == sj.SJ_OK
    E2 = r64(F(eps) * F(eps))
    w = eps * (1.0 + 2.0 ** -16)
    inv_w = 1.0 / w
    ng = [int(math.floor((gmax[j] - gmin[j]) / w)) + 1 for j in range(d)]
    # the band is narrow: its width relative to eps^2 grows with the FP32
    # rounding of the stored coordinates, u * (range / eps)
    X = float(np.max(gmax - gmin))
    assert (hi - max(lo, 0.0)) / float(E2) < 1e-4 + 40 * 2.0 ** -24 * X / eps
    checked = 0
    for k, p in enumerate(pts):
        cells = [cell_of(p[j], gmin[j], inv_w, ng[j]) for j in range(d)]
        for q in extra[7 * k: 7 * k + 7]:
            cq = [cell_of(q[j], gmin[j], inv_w, ng[j]) for j in range(d)]
            if max(abs(a - b) for a, b in zip(cells, cq)) > 1:
                continue           # not adjacent: never compared
            s = kernel_s32(p, q, gmin, w32, cells)
            mem = exact_member(p, q, E2)
            if s <= F(lo):
                assert mem, (d, k)
            if s > F(hi):
                assert not mem, (d, k)
            checked += 1
    assert checked > 100


def test_margin_rejects_unusable_grids():
    # a grid many orders of magnitude wider than eps leaves no useful margin
    st, _, _, _ = sj.sj_fp32_margin(2, 1e-9, np.array([0.0, 0.0]), np.array([1e8, 1.0]))
    assert st in (sj.SJ_ERANGE,)
    st, _, _, _ = sj.sj_fp32_margin(2, -1.0, np.zeros(2), np.ones(2))
    assert st == sj.SJ_EINVAL


# ---------------------------------------------------------------- cell frame

def rec_cell(x, gmin, w, inv_w, ng):
    """The cell-frame record of one coordinate and its cell: y =
    fl32(fl64(fl64(x - g_min) - fl64(4 K w))), K = floor(c / 4)."""
    a = r64(F(x) - F(gmin))
    c = min(max(int(math.floor(r64(a * F(inv_w)))), 0), ng - 1)
    T = r64(F(4 * (c >> 2)) * F(w))
    return r32(r64(a - T)), c


def kernel_s32_cell(p, q, gmin, w, w32, inv_w, ng):
    """s32 as the kernel computes it on cell-frame records: the home cell
    centre within the four-cell frame, the candidate moved by whole frame
    steps k = rint(z / (4 w32)) (ties to even), then the same expanded sum
    as in the grid frame.  Returns (s32, number of frame steps taken)."""
    d = len(p)
    inv4 = r32(r64(F(1) / (4 * F(w32))))
    zp, zq, steps = [], [], 0
    for j in range(d):
        yp, cp = rec_cell(p[j], gmin[j], w, inv_w, ng[j])
        yq, _ = rec_cell(q[j], gmin[j], w, inv_w, ng[j])
        o = r32(r32(F(cp & 3) + F(1, 2)) * F(w32))
        zp.append(r32(yp - o))
        zr = r32(yq - o)
        k = round(r32(zr * inv4))            # round half to even, like rintf
        steps += k != 0
        zq.append(r32(-(4 * F(w32)) * k + zr))
    pp = F(0)
    qq = F(0)
    for j in range(d):
        pp = r32(zp[j] * zp[j] + pp)
        qq = r32(zq[j] * zq[j] + qq)
    acc = r32(qq + pp)
    for j in range(d):
        acc = r32((-2 * zp[j]) * zq[j] + acc)
    return acc, steps


@pytest.mark.parametrize("d,eps,scale,offset", [
    (2, 0.5, 1e7, 0.0), (3, 1.0, 1e6, 1e9), (2, 0.31915, 100.0, 0.0), (6, 13.55112, 100.0, 0.0),
    (8, 0.9, 10.0, 5.0), (1, 1e-3, 1e5, -3e5), (4, 2e-4, 4e4, 0.0)])
def test_cell_frame_margin_sound_on_threshold_pairs(d, eps, scale, offset):
    rng = np.random.default_rng(int(scale) % 1000 + 31 * d)
    w = eps * (1.0 + 2.0 ** -16)
    pts = offset + rng.uniform(0, scale, size=(60, d))
    # half of the points sit just below a four-cell frame boundary in
    # dimension 0, so that their partners fall into the next frame
    g0 = float(np.min(pts[:, 0])) - eps
    for p in pts[::2]:
        c = int((p[0] - g0) / w)
        p[0] = g0 + (4 * (c // 4) + 4) * w - 0.3 * eps
    extra = []
    for p in pts:
        v = rng.normal(size=d)
        v /= np.linalg.norm(v)
        v[0] = abs(v[0])
        for f in (1.0, 1.0 + 2.0 ** -52, 1.0 - 2.0 ** -52, 1.0 + 3e-7, 1.0 - 3e-7,
                  1.0 + 2e-6, 1.0 - 2e-6):
            extra.append(p + v * eps * f)
    allp = np.concatenate([pts, np.array(extra)])
    gmin = allp.min(axis=0) - eps
    gmax = allp.max(axis=0) + eps
    st, w32, lo, hi = sj.sj_fp32_margin_frame(d, eps, gmin, gmax, sj.SJ_FRAME_CELL)
    assert st == sj.SJ_OK
    E2 = r64(F(eps) * F(eps))
    inv_w = 1.0 / w
    ng = [int(math.floor((gmax[j] - gmin[j]) / w)) + 1 for j in range(d)]
    # the band does not grow with the extent of the grid
    assert (hi - max(lo, 0.0)) / float(E2) < 2000 * 2.0 ** -24
    checked = stepped = 0
    for k, p in enumerate(pts):
        cells = [rec_cell(p[j], gmin[j], w, inv_w, ng[j])[1] for j in range(d)]
        for q in extra[7 * k: 7 * k + 7]:
            cq = [rec_cell(q[j], gmin[j], w, inv_w, ng[j])[1] for j in range(d)]
            if max(abs(a - b) for a, b in zip(cells, cq)) > 1:
                continue
            for a, b, ca, cb in ((p, q, cells, cq), (q, p, cq, cells)):
                s, steps = kernel_s32_cell(a, b, gmin, w, w32, inv_w, ng)
                mem = exact_member(a, b, E2)
                if s <= F(lo):
                    assert mem, (d, k)
                if s > F(hi):
                    assert not mem, (d, k)
                stepped += steps > 0
                checked += 1
    assert checked > 200
    assert stepped > 20      # pairs across a frame boundary were exercised


def test_cell_frame_exact_difference_across_frames():
    """On coordinates exact in FP32 (multiples of 2^-8 and w a power of 2)
    every step above is exact, so the kernel's z_p - z_q must equal x_p - x_q
    exactly, also when q lies in the neighbouring four-cell frame and the
    grid is 2^30 cells wide."""
    eps = 2.0 ** -3 * (1.0 - 2.0 ** -20)
    w = eps * (1.0 + 2.0 ** -16)
    gmin = 0.0
    ng = 2 ** 30
    inv_w = 1.0 / w
    for c in (3, 7, 4 * 12345 + 3, 2 ** 29 + 3, 2 ** 30 - 5):
        x = (c + 0.75) * w
        x = float(F(x).limit_denominator(2 ** 40))
        for dx in (0.3 * eps, 0.9 * eps, -0.8 * eps):
            y = x + dx
            yp, cp = rec_cell(x, gmin, w, inv_w, ng)
            yq, cq = rec_cell(y, gmin, w, inv_w, ng)
            w32 = r32(F(w))
            o = r32(r32(F(cp & 3) + F(1, 2)) * w32)
            inv4 = r32(r64(F(1) / (4 * w32)))
            zr = r32(yq - o)
            k = round(r32(zr * inv4))
            assert k == -((cq >> 2) - (cp >> 2))
            zq = r32(-(4 * w32) * k + zr)
            assert zq == zr - 4 * w32 * k           # the frame step is exact
            zp = r32(yp - o)
            assert abs(float(zp - zq) + dx) < 8 * 2.0 ** -24 * w + 4 * abs(c) * 2.0 ** -53 * w


def test_cell_frame_margin_at_any_extent():
    # the grid frame gives up on wide grids; the cell frame keeps a narrow band
    for d, X in ((1, 1e8), (2, 1e8), (3, 5e8), (8, 1e7)):
        gmin, gmax = np.zeros(d), np.full(d, X)
        st0, _, _, _ = sj.sj_fp32_margin_frame(d, 1.0, gmin, gmax, sj.SJ_FRAME_GRID)
        st1, _, lo, hi = sj.sj_fp32_margin_frame(d, 1.0, gmin, gmax, sj.SJ_FRAME_CELL)
        assert st0 == sj.SJ_ERANGE
        assert st1 == sj.SJ_OK and 0.0 < lo < 1.0 < hi and hi - lo < 2000 * 2.0 ** -24
    st, _, _, _ = sj.sj_fp32_margin_frame(2, 1.0, np.zeros(2), np.ones(2), 7)
    assert st == sj.SJ_EINVAL
    # where the grid frame is tight both frames give similar bands
    st0, _, lo0, hi0 = sj.sj_fp32_margin_frame(3, 2.0, np.zeros(3), np.full(3, 100.0), sj.SJ_FRAME_GRID)
    st1, _, lo1, hi1 = sj.sj_fp32_margin_frame(3, 2.0, np.zeros(3), np.full(3, 100.0), sj.SJ_FRAME_CELL)
    assert st0 == st1 == sj.SJ_OK and hi1 - lo1 < hi0 - lo0


# ---------------------------------------------------------------- difference form (d > 8)

def kernel_s32_diff(p, q, fmin, chains=2):
    """s32 of the high-dimensional kernel: fma chains of fl32(y_p - y_q)^2,
    coordinate j in chain j mod chains, the chains added at the end (the
    kernel uses two; one chain is the plain sequential sum)."""
    acc = [F(0)] * chains
    for j in range(len(p)):
        yp = r32(r64(F(p[j]) - F(fmin[j])))
        yq = r32(r64(F(q[j]) - F(fmin[j])))
        t = r32(yp - yq)
        acc[j % chains] = r32(t * t + acc[j % chains])
    s = acc[0]
    for a in acc[1:]:
        s = r32(s + a)
    return s


@pytest.mark.parametrize("d,eps,scale,offset", [
    (9, 30.0, 100.0, 0.0), (12, 0.7, 1000.0, -50.0), (16, 55.0, 100.0, 0.0), (3, 0.37, 30.0, 1e5)])
def test_difference_form_margin_sound_on_threshold_pairs(d, eps, scale, offset):
    rng = np.random.default_rng(int(eps * 100) + d)
    pts = offset + rng.uniform(0, scale, size=(50, d))
    extra = []
    for p in pts:
        v = rng.normal(size=d)
        v /= np.linalg.norm(v)
        for f in (1.0, 1.0 + 2.0 ** -52, 1.0 - 2.0 ** -52, 1.0 + 3e-7, 1.0 - 3e-7,
                  1.0 + 2e-6, 1.0 - 2e-6, 0.5, 1.7):
            extra.append(p + v * eps * f)
    allp = np.concatenate([pts, np.array(extra)])
    fmin = allp.min(axis=0) - eps
    fmax = allp.max(axis=0) + eps
    st, lo, hi = sj.sj_fp32_margin_diff(d, eps, fmin, fmax)
    assert st == sj.SJ_OK
    E2 = r64(F(eps) * F(eps))
    X = float(np.max(fmax - fmin))
    assert 0.0 < lo < float(E2) < hi
    assert (hi - lo) / float(E2) < 1e-4 + 40 * 2.0 ** -24 * X / eps
    checked = 0
    for k, p in enumerate(pts):
        for q in extra[9 * k: 9 * k + 9]:
            mem = exact_member(p, q, E2)
            for chains in (2, 1):
                s = kernel_s32_diff(p, q, fmin, chains)
                if s <= F(lo):
                    assert mem, (d, k, chains)
                if s > F(hi):
                    assert not mem, (d, k, chains)
            checked += 1
    assert checked == 450


def test_difference_form_margin_arguments():
    st, _, _ = sj.sj_fp32_margin_diff(17, 1.0, np.zeros(17), np.ones(17))
    assert st == sj.SJ_EINVAL
    st, _, _ = sj.sj_fp32_margin_diff(10, 1e-9, np.zeros(10), np.full(10, 1e8))
    assert st == sj.SJ_ERANGE


# ---------------------------------------------------------------- expanded form (d > 8)

def kernel_s32_hd(p, q, fmin, w32, cells, grid, mid):
    """s32 of the high-dimensional kernel's expanded form: z_j = fl32(y_j -
    o_j) about the home cell centre in a grid dimension and mid[j] in the
    others; |z|^2 as fma chains; fl(qq + pp) starts the chain of the even
    coordinates' terms m_j z_q,j, the odd ones form a second chain, and the
    two are added at the end."""
    d = len(p)
    zp, zq = [], []
    for j in range(d):
        o = r32(r32(F(cells[j]) + F(1, 2)) * F(w32)) if grid[j] else F(float(mid[j]))
        yp = r32(r64(F(p[j]) - F(fmin[j])))
        yq = r32(r64(F(q[j]) - F(fmin[j])))
        zp.append(r32(yp - o))
        zq.append(r32(yq - o))
    pp = qq = F(0)
    for j in range(d):
        pp = r32(zp[j] * zp[j] + pp)
        qq = r32(zq[j] * zq[j] + qq)
    acc = [r32(qq + pp), F(0)]
    for j in range(d):
        acc[j % 2] = r32((-2 * zp[j]) * zq[j] + acc[j % 2])
    return r32(acc[0] + acc[1])


@pytest.mark.parametrize("d,eps,scale,offset", [
    (9, 30.0, 100.0, 0.0), (12, 20.0, 100.0, -50.0), (16, 55.0, 100.0, 0.0), (16, 66.2, 100.0, 1e3)])
def test_expanded_form_hd_margin_sound_on_threshold_pairs(d, eps, scale, offset):
    rng = np.random.default_rng(int(eps * 10) + d)
    pts = offset + rng.uniform(0, scale, size=(40, d))
    extra = []
    for p in pts:
        v = rng.normal(size=d)
        v /= np.linalg.norm(v)
        for f in (1.0, 1.0 + 2.0 ** -52, 1.0 - 2.0 ** -52, 1.0 + 3e-7, 1.0 - 3e-7,
                  1.0 + 2e-6, 1.0 - 2e-6, 0.5):
            extra.append(p + v * eps * f)
    allp = np.concatenate([pts, np.array(extra)])
    fmin = allp.min(axis=0) - eps
    fmax = allp.max(axis=0) + eps
    grid = np.zeros(d, dtype=np.int32)
    grid[rng.choice(d, size=6, replace=False)] = 1
    st, lo, hi, mid = sj.sj_fp32_margin_hd(d, eps, fmin, fmax, grid)
    assert st == sj.SJ_OK
    E2 = r64(F(eps) * F(eps))
    assert 0.0 < lo < float(E2) < hi
    # the band grows with the extent of the dimensions outside the grid
    X = float(np.max(fmax - fmin))
    assert (hi - lo) / float(E2) < 1e-4 + 200 * d * 2.0 ** -24 * (X / eps) ** 2
    for j in range(d):
        if not grid[j]:
            assert mid[j] == np.float32(0.5 * (fmax[j] - fmin[j]))
    w = eps * (1.0 + 2.0 ** -16)
    inv_w = 1.0 / w
    w32 = float(np.float32(w))
    ng = [int(math.floor((fmax[j] - fmin[j]) / w)) + 1 for j in range(d)]
    checked = 0
    for k, p in enumerate(pts):
        cells = [cell_of(p[j], fmin[j], inv_w, ng[j]) if grid[j] else 0 for j in range(d)]
        for q in extra[8 * k: 8 * k + 8]:
            cq = [cell_of(q[j], fmin[j], inv_w, ng[j]) if grid[j] else 0 for j in range(d)]
            if max(abs(a - b) for a, b in zip(cells, cq)) > 1:
                continue           # not adjacent in the grid: never compared
            s = kernel_s32_hd(p, q, fmin, w32, cells, grid, mid)
            mem = exact_member(p, q, E2)
            if s <= F(lo):
                assert mem, (d, k)
            if s > F(hi):
                assert not mem, (d, k)
            checked += 1
    assert checked > 100


def test_expanded_form_hd_margin_arguments():
    g = np.ones(17, dtype=np.int32)
    st, _, _, _ = sj.sj_fp32_margin_hd(17, 1.0, np.zeros(17), np.ones(17), g)
    assert st == sj.SJ_EINVAL
    # a data range far wider than eps outside the grid leaves no usable band
    g = np.zeros(10, dtype=np.int32)
    g[:6] = 1
    st, _, _, _ = sj.sj_fp32_margin_hd(10, 1e-3, np.zeros(10), np.full(10, 1e6), g)
    assert st == sj.SJ_ERANGE
