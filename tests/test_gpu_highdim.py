"""Points of more than 8 dimensions (up to 16): the grid covers the six
dimensions with the most cells, the search refines on every coordinate.
Results are compared with the definition (brute force)."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1803_04120_gb300 import datagen, sj

pytestmark = pytest.mark.gpu


def keys(pairs):
    return np.sort(sj.pairs_to_keys(pairs))


def eps_for(n, d, k, side=100.0):
    return (k * side ** d / (n * datagen.ball_volume(d))) ** (1.0 / d)


def clustered(n, d, seed, side=100.0, sigma=2.0, per=60):
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0, side, size=(max(1, n // per), d))
    pts = centres[rng.integers(0, len(centres), n)] + rng.normal(0, sigma, size=(n, d))
    pts[: n // 10] = rng.uniform(0, side, size=(n // 10, d))
    return pts


@pytest.mark.parametrize("d", [9, 12, 16])
def test_highdim_matches_bruteforce(d):
    rng = np.random.default_rng(400 + d)
    cases = [(rng.uniform(0, 100, size=(3000, d)), eps_for(3000, d, 20)),
             (clustered(5000, d, 500 + d), 4.0)]
    # the uniform case takes the expanded-form sum, the clustered one (small
    # eps against the data range) the difference form
    assert [hd_form(p, e) for p, e in cases] == ["expanded", "difference"]
    for pts, eps in cases:
        want = orc.bruteforce(pts, eps)
        for prec in (sj.SJ_PREC_FP32_RECHECK, sj.SJ_PREC_FP64):
            for uni in (True, False):
                for lookup in (sj.SJ_LOOKUP_AUTO, sj.SJ_LOOKUP_SEARCH, sj.SJ_LOOKUP_COORDS):
                    with sj.Context(prec=prec, unicomp=uni, lookup=lookup) as ctx:
                        got = keys(ctx.sj_selfjoin(pts, eps))
                        st = ctx.sj_last_stats()
                    assert np.array_equal(got, np.sort(want)), (d, prec, uni, lookup, len(got), len(want))
                    assert st["frame"] == (0 if prec == sj.SJ_PREC_FP32_RECHECK else -1)
        assert len(want) > len(pts)


def hd_form(pts, eps):
    """'expanded' or 'difference': the FP32 sum the index chooses (the
    expanded form while its band is below 2^-10 eps^2, as the library
    decides from the same margins), for the six dimensions with the most
    cells as the grid."""
    d = pts.shape[1]
    fmin = pts.min(axis=0) - eps
    fmax = pts.max(axis=0) + eps
    w = eps * (1.0 + 2.0 ** -16)
    cells = np.floor((fmax - fmin) / w) + 1.0
    grid = np.zeros(d, dtype=np.int32)
    taken = []
    for _ in range(6):
        best = max((j for j in range(d) if j not in taken), key=lambda j: (cells[j], -j))
        taken.append(best)
    grid[taken] = 1
    est, elo, ehi, _ = sj.sj_fp32_margin_hd(d, eps, fmin, fmax, grid)
    dst, _, _ = sj.sj_fp32_margin_diff(d, eps, fmin, fmax)
    narrow = est == sj.SJ_OK and ehi - max(elo, 0.0) <= eps * eps * 2.0 ** -10
    return "expanded" if est == sj.SJ_OK and (narrow or dst != sj.SJ_OK) else "difference"


@pytest.mark.parametrize("eps,form", [(3.0, "difference"), (30.0, "expanded")])
def test_highdim_band_pairs_are_rechecked(eps, form):
    rng = np.random.default_rng(410)
    d = 11
    base = rng.uniform(0, 40, size=(600, d))
    extra = []
    for p in base:
        v = rng.normal(size=d)
        v /= np.linalg.norm(v)
        f = 1.0 + float(rng.integers(-4, 5)) * 2.0 ** -52
        if rng.random() < 0.5:
            f = 1.0 + float(rng.choice([-3, -1, 0, 1, 3])) * 2.0 ** -24 * float(rng.random())
        extra.append(p + v * eps * f)
    pts = np.concatenate([base, np.array(extra)])
    assert hd_form(pts, eps) == form
    want = np.sort(orc.bruteforce(pts, eps))
    with sj.Context() as ctx:
        assert np.array_equal(keys(ctx.sj_selfjoin(pts, eps)), want)
        assert ctx.sj_last_stats()["rechecks"] > 0


def test_highdim_grid_dims_batching_and_device_path():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(420)
    d = 12
    pts = rng.uniform(0, 100, size=(6000, d))
    pts[:, [1, 4, 7]] *= 0.01           # narrow dimensions: fewest cells, not in the grid
    pts[:, [1, 4, 7]] += 3.0
    eps = 9.0
    want = np.sort(orc.bruteforce(pts, eps))
    # host result in many small batches
    with sj.Context(out_cap_bytes=256 << 10, min_batches=5) as ctx:
        assert np.array_equal(keys(ctx.sj_selfjoin(pts, eps)), want)
        assert ctx.sj_last_stats()["batches"] >= 5
        idx = ctx.sj_build_index(pts, eps)
        info = idx.sj_index_info()
        assert info["d"] == d and info["grid_d"] == 6
        assert not set(info["grid_dim"]) & {1, 4, 7}
        assert info["grid_dim"] == sorted(info["grid_dim"])
        B, G, A, M = idx.sj_index_export()
        assert G[-1] == len(pts) and np.array_equal(np.sort(A), np.arange(len(pts)))
        assert np.array_equal(keys(ctx.sj_selfjoin_index(idx)), want)
        idx.free()
    # device-resident, count first, then an exact-size buffer
    with sj.Context() as ctx:
        dp = torch.from_numpy(pts).cuda()
        n = ctx.sj_selfjoin_count(dp, eps)
        assert n == len(want)
        out = torch.empty((n, 2), dtype=torch.int32, device="cuda")
        assert ctx.sj_selfjoin_device(dp, eps, out) == n
        assert np.array_equal(keys(out.cpu().numpy().view(np.uint32)), want)


def test_highdim_wide_range_and_limits():
    rng = np.random.default_rng(430)
    d = 10
    pts = rng.uniform(0, 3.0, size=(2000, d))
    pts[:, 0] *= 2e6                     # range / eps beyond the FP32 margin: FP64 arithmetic
    pts[:200, 0] = rng.uniform(1e6, 1e6 + 2.0, 200)
    eps = 1.0
    st, _, _ = sj.sj_fp32_margin_diff(d, eps, pts.min(axis=0) - eps, pts.max(axis=0) + eps)
    assert st == sj.SJ_ERANGE
    with sj.Context() as ctx:
        assert np.array_equal(keys(ctx.sj_selfjoin(pts, eps)), np.sort(orc.bruteforce(pts, eps)))
        assert ctx.sj_last_stats()["frame"] == -1
        with pytest.raises(sj.SJError) as ei:
            ctx.sj_selfjoin(np.zeros((4, 17)), 1.0)
        assert ei.value.status == sj.SJ_EINVAL
        with pytest.raises(sj.SJError) as ei:
            ctx.sj_join2_device(pts, pts, 1.0, None)
        assert ei.value.status == sj.SJ_EINVAL
        res = ctx.sj_selfjoin_multi([(pts, 1.0), (pts[:, :3].copy(), 0.5)], raise_errors=False)
        assert ctx.last_multi_status == [sj.SJ_EINVAL, sj.SJ_OK] and res[0] is None


@pytest.mark.parametrize("d,m", [(10, 2), (12, 2), (9, 3)])
def test_highdim_unit_lattice_closed_form(d, m):
    # spacing 1, eps = 1: every point, itself and its axis neighbours
    pts = np.stack(np.meshgrid(*[np.arange(m, dtype=np.float64)] * d, indexing="ij"), -1).reshape(-1, d)
    total = m ** d + 2 * d * (m - 1) * m ** (d - 1)
    for prec in (sj.SJ_PREC_FP32_RECHECK, sj.SJ_PREC_FP64):
        for uni in (True, False):
            with sj.Context(prec=prec, unicomp=uni) as ctx:
                assert len(ctx.sj_selfjoin(pts, 1.0)) == total, (d, m, prec, uni)
