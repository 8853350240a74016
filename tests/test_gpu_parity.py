"""Parity of the CUDA self-join with the CPU oracle (GPU required).

Every comparison is element-by-element on sorted (i << 32) | j keys: the
result must equal the oracle's exactly, in both precision modes, with and
without UNICOMP, through every entry point.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1803_04120_gb300 import datagen, sj

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
MODES = [(sj.SJ_PREC_FP32_RECHECK, True), (sj.SJ_PREC_FP64, True),
         (sj.SJ_PREC_FP32_RECHECK, False), (sj.SJ_PREC_FP64, False)]
# dense table, binary search of B, binary search of coordinate tuples
LOOKUPS = (sj.SJ_LOOKUP_AUTO, sj.SJ_LOOKUP_SEARCH, sj.SJ_LOOKUP_COORDS)


@pytest.fixture(scope="module")
def ctxs():
    out = {}
    for prec, uni in MODES:
        for lookup in LOOKUPS:
            out[(prec, uni, lookup)] = sj.Context(prec=prec, unicomp=uni, lookup=lookup)
    yield out
    for c in out.values():
        c.close()


def gpu_keys(ctx, pts, eps):
    return sj.pairs_to_keys(ctx.sj_selfjoin(pts, eps))


def assert_same(got, want, what=""):
    if got.shape != want.shape or not np.array_equal(got, want):
        gs, ws = set(got.tolist()), set(want.tolist())
        missing = sorted(ws - gs)[:5]
        extra = sorted(gs - ws)[:5]
        dup = got.size - len(gs)
        pytest.fail(f"{what}: got {got.size} want {want.size}; missing {[(k >> 32, k & 0xffffffff) for k in missing]} "
                    f"extra {[(k >> 32, k & 0xffffffff) for k in extra]} duplicates {dup}")


# ------------------------------------------------------------------ small cases

@pytest.mark.parametrize("prec,uni", MODES)
def test_config1_equals_bruteforce(ctxs, prec, uni):
    cfg = datagen.CONFIG1
    pts = datagen.make_points(cfg)
    want = orc.bruteforce(pts, cfg["eps"])
    for lookup in LOOKUPS:
        got = gpu_keys(ctxs[(prec, uni, lookup)], pts, cfg["eps"])
        assert_same(got, want, f"config1 prec={prec} unicomp={uni} lookup={lookup}")


@pytest.mark.parametrize("d", [1, 2, 3, 4, 5, 6, 7, 8])
def test_random_all_dims_all_modes(ctxs, d):
    rng = np.random.default_rng(1000 + d)
    for trial in range(3):
        n = int(rng.integers(50, 3000))
        pts = rng.uniform(-10, 10, size=(n, d))
        if trial == 1:
            pts[n // 3: 2 * n // 3] = pts[: 2 * n // 3 - n // 3]   # duplicates
        vol = 20.0 ** d
        k = float(rng.choice([4.0, 40.0, 400.0]))
        eps = (k * vol / (n * datagen.ball_volume(d))) ** (1.0 / d)
        want = orc.grid_join(pts, eps)
        for key, ctx in ctxs.items():
            got = gpu_keys(ctx, pts, eps)
            assert_same(got, want, f"d={d} trial={trial} n={n} eps={eps} mode={key}")


def test_heavy_cell_spans_many_items_and_chunks(ctxs):
    # one cell with 3000 points (many query blocks and candidate chunks) plus
    # a sparse background
    rng = np.random.default_rng(5)
    dense = rng.uniform(0, 0.2, size=(3000, 2))
    bg = rng.uniform(0, 50, size=(500, 2))
    pts = np.concatenate([dense, bg])
    eps = 0.25
    want = orc.grid_join(pts, eps)
    for key, ctx in ctxs.items():
        assert_same(gpu_keys(ctx, pts, eps), want, f"heavy cell {key}")


def test_edge_cases(ctxs):
    ctx = ctxs[(sj.SJ_PREC_FP32_RECHECK, True, sj.SJ_LOOKUP_AUTO)]
    # a single point
    one = np.array([[1.0, 2.0, 3.0]])
    assert_same(gpu_keys(ctx, one, 0.5), np.array([0], dtype=np.uint64), "n=1")
    # all points identical: n^2 pairs
    same = np.full((100, 4), 7.25)
    assert gpu_keys(ctx, same, 1e-9).size == 100 * 100
    # eps larger than the data range: all pairs
    pts = datagen.uniform(300, 3, seed=9)
    assert gpu_keys(ctx, pts, 1000.0).size == 300 * 300
    # eps small against the data range: self-pairs only
    k = gpu_keys(ctx, pts, 1e-4)
    assert_same(k, (np.arange(300, dtype=np.uint64) << np.uint64(32)) | np.arange(300, dtype=np.uint64), "tiny eps")
    # 2^31 or more cells in one dimension are refused, not approximated
    with pytest.raises(sj.SJError) as ei:
        ctx.sj_selfjoin(pts, 1e-12)
    assert ei.value.status == sj.SJ_ERANGE
    # 1e24 cells: coordinate-tuple order, self-pairs only
    assert_same(gpu_keys(ctx, pts, 1e-6), k, "1e24-cell grid")
    assert ctx.sj_selfjoin(pts, 1e-4).shape[0] == 300
    # negative and large-offset coordinates
    off = datagen.uniform(2000, 2, seed=10) - 1e6
    assert_same(gpu_keys(ctx, off, 0.7), orc.grid_join(off, 0.7), "offset coordinates")


@pytest.mark.parametrize("d,m", [(2, 30), (3, 12), (4, 7)])
def test_unit_lattice_closed_form_gpu(ctxs, d, m):
    axes = [np.arange(m, dtype=np.float64)] * d
    pts = np.stack([g.ravel() for g in np.meshgrid(*axes, indexing="ij")], axis=1)
    expect = m ** d + 2 * d * (m - 1) * m ** (d - 1)
    for key, ctx in ctxs.items():
        assert gpu_keys(ctx, pts, 1.0).size == expect, key
        assert gpu_keys(ctx, pts, 1.0 - 2.0 ** -40).size == m ** d, key


def test_fma_contraction_detector_gpu(ctxs):
    # fl(fl(a0^2) + fl(a1^2)) > fl(eps^2) >= fma(a1, a1, fl(a0^2)): not a member
    pts = np.array([[0.9433567169983137, 0.6489745531369242], [0.0, 0.0]])
    eps = 1.1450283254684606
    for key, ctx in ctxs.items():
        got = gpu_keys(ctx, pts, eps)
        assert_same(got, np.array([0, (1 << 32) | 1], dtype=np.uint64), f"fma detector {key}")


def test_adversarial_band_pairs(ctxs):
    # pairs at squared distance E2 * (1 +- k 2^-24) and +- a few FP64 ulps:
    # inside the FP32 margin, so the FP64 recheck must decide them
    rng = np.random.default_rng(77)
    for d in (2, 3, 6):
        eps = 0.37
        base = rng.uniform(0, 30, size=(400, d))
        extra = []
        for p in base:
            v = rng.normal(size=d)
            v /= np.linalg.norm(v)
            f = 1.0 + float(rng.choice([-3, -1, 0, 1, 3])) * 2.0 ** -24 * float(rng.random())
            if rng.random() < 0.5:
                f = 1.0 + float(rng.integers(-4, 5)) * 2.0 ** -52
            extra.append(p + v * eps * f)
        pts = np.concatenate([base, np.array(extra)])
        want = orc.grid_join(pts, eps)
        for key, ctx in ctxs.items():
            assert_same(gpu_keys(ctx, pts, eps), want, f"band d={d} {key}")
        st = ctxs[(sj.SJ_PREC_FP32_RECHECK, True, sj.SJ_LOOKUP_AUTO)]
        st.sj_selfjoin(pts, eps)
        assert st.sj_last_stats()["rechecks"] > 0


def test_cell_boundary_plants(ctxs):
    rng = np.random.default_rng(8)
    for d in (2, 3, 5):
        eps = 0.3
        base = rng.uniform(0, 3, size=(200, d))
        extra = []
        for p in base:
            k = int(rng.integers(0, d))
            for f in (1.0, 1.0 + 2.0 ** -52, 1.0 - 2.0 ** -52):
                q = p.copy()
                q[k] += eps * f
                extra.append(q)
        pts = np.concatenate([base, np.array(extra)])
        want = orc.bruteforce(pts, eps)
        for key, ctx in ctxs.items():
            assert_same(gpu_keys(ctx, pts, eps), want, f"boundary d={d} {key}")


# ------------------------------------------------------------------ entry points

def test_device_entry_point_and_overflow():
    torch = pytest.importorskip("torch")
    pts = datagen.uniform(5000, 3, seed=12)
    eps = 3.0
    want = orc.grid_join(pts, eps)
    with sj.Context() as ctx:
        d_pts = torch.from_numpy(pts).cuda()
        out = torch.empty((want.size + 10, 2), dtype=torch.int32, device="cuda")
        n = ctx.sj_selfjoin_device(d_pts, eps, out)
        assert n == want.size
        got = sj.pairs_to_keys(out[:n].cpu().numpy().view(np.uint32))
        assert_same(got, want, "device entry point")
        # host points through the device entry point
        n2 = ctx.sj_selfjoin_device(pts, eps, out)
        assert n2 == want.size
        # too small: the count is still reported
        small = torch.empty((100, 2), dtype=torch.int32, device="cuda")
        with pytest.raises(sj.SJError) as ei:
            ctx.sj_selfjoin_device(d_pts, eps, small)
        assert ei.value.status == sj.SJ_EOVERFLOW
        assert ctx.sj_selfjoin_device(d_pts, eps, small, raise_overflow=False) == want.size
        assert ctx.sj_selfjoin_count(d_pts, eps) == want.size
        st = ctx.sj_last_stats()
        assert st["evaluations"] > 0


def test_device_points_read_in_place():
    """Calls whose index ends with them read device points in place (no
    copy): a view that starts one row into a larger tensor (8-byte but not
    256-byte aligned) joins like the oracle, and no call writes the caller's
    array; the persistent index (sj_build_index) keeps its own copy, so a
    later change of the array does not reach it."""
    torch = pytest.importorskip("torch")
    pts = datagen.uniform(6001, 4, seed=13)
    eps = 4.0
    want = orc.grid_join(pts[1:], eps)
    big = torch.from_numpy(pts).cuda()
    view = big[1:]
    assert view.data_ptr() % 256 != 0
    before = big.clone()
    with sj.Context() as ctx:
        out = torch.empty((want.size + 10, 2), dtype=torch.int32, device="cuda")
        n = ctx.sj_selfjoin_device(view, eps, out)
        assert n == want.size
        assert_same(sj.pairs_to_keys(out[:n].cpu().numpy().view(np.uint32)), want, "row-offset view")
        assert ctx.sj_selfjoin_count(view, eps) == want.size
        assert_same(sj.pairs_to_keys(ctx.sj_selfjoin(view, eps)), want, "host result from device points")
        assert torch.equal(big, before)
        idx = ctx.sj_build_index(view, eps)
        big.fill_(0.0)          # the index holds its own copy of the points
        assert_same(sj.pairs_to_keys(ctx.sj_selfjoin_index(idx)), want, "index after the array changed")
        idx.free()


def test_batching_small_cap_many_batches_and_retries():
    pts = datagen.uniform(20000, 2, seed=13)
    eps = 1.5
    want = orc.grid_join(pts, eps)
    for cap in (1 << 16, 1 << 18, 1 << 20):
        with sj.Context(out_cap_bytes=cap, sorted=True) as ctx:
            got = ctx.sj_selfjoin(pts, eps)
            k = (got[:, 0].astype(np.uint64) << np.uint64(32)) | got[:, 1].astype(np.uint64)
            assert np.all(np.diff(k.view(np.int64)) > 0), "sorted output"
            assert_same(k, want, f"cap={cap}")
            st = ctx.sj_last_stats()
            assert st["batches"] >= 3


def test_stream_entry_point():
    pts = datagen.uniform(20000, 3, seed=14)
    eps = 2.5
    want = orc.grid_join(pts, eps)
    chunks = []
    with sj.Context(out_cap_bytes=1 << 20) as ctx:
        ctx.sj_selfjoin_stream(pts, eps, lambda a: chunks.append(a) and False)
    got = sj.pairs_to_keys(np.concatenate(chunks))
    assert len(chunks) >= 3
    assert_same(got, want, "stream")


def test_index_reuse_and_worked_example():
    fx = json.load(open(os.path.join(GOLDEN, "worked_example_sec4d.json")))
    pts = np.array(fx["points"])
    paper = fx["paper"]
    with sj.Context() as ctx:
        ix = ctx.sj_build_index(pts, fx["eps"])
        info = ix.sj_index_info()
        assert info["ng"] == paper["cells_per_dim"]
        assert info["n_cells"] == paper["non_empty_cells"]
        B, G, A, M = ix.sj_index_export()
        assert B.tolist() == fx["constructed"]["non_empty_linear_ids"]
        h6 = paper["C6_linear_id"]
        h = B.tolist().index(h6)
        assert h + 1 == 6
        assert sorted(A[G[h]:G[h + 1]].tolist()) == sorted(paper["C6_points"])
        assert B.tolist().index(paper["query_cell_linear_id"]) + 1 == paper["query_cell_rank_1based"]
        # M_1: column 3 empty, the others occupied; M_2: all rows occupied
        assert [(int(M[0, 0]) >> c) & 1 for c in range(7)] == [1, 1, 1, 0, 1, 1, 1]
        assert [(int(M[1, 0]) >> c) & 1 for c in range(7)] == [1] * 7
        # G tiles [0, n) and A is a permutation
        assert G[0] == 0 and G[-1] == len(pts) and np.all(np.diff(G.astype(np.int64)) > 0)
        assert sorted(A.tolist()) == list(range(len(pts)))
        want = orc.bruteforce(pts, fx["eps"])
        assert_same(sj.pairs_to_keys(ctx.sj_selfjoin_index(ix)), want, "index reuse")
        assert_same(sj.pairs_to_keys(ctx.sj_selfjoin_index(ix)), want, "index reuse twice")
        ix.free()


def test_invalid_arguments():
    with sj.Context() as ctx:
        pts = np.zeros((10, 2))
        for bad_eps in (0.0, -1.0, float("nan"), float("inf")):
            with pytest.raises(sj.SJError) as ei:
                ctx.sj_selfjoin(pts, bad_eps)
            assert ei.value.status == sj.SJ_EINVAL
        bad = pts.copy()
        bad[3, 1] = np.nan
        with pytest.raises(sj.SJError) as ei:
            ctx.sj_selfjoin(bad, 1.0)
        assert ei.value.status == sj.SJ_EINVAL
        with pytest.raises(sj.SJError) as ei:
            ctx.sj_selfjoin(np.zeros((4, 17)), 1.0)
        assert ei.value.status == sj.SJ_EINVAL
        # the context stays usable after errors
        assert ctx.sj_selfjoin(pts, 1.0).shape[0] == 100


def test_unicomp_halves_evaluations():
    pts = datagen.uniform(50000, 3, seed=15)
    eps = datagen.eps_for_neighbors(50000, 3, 32, side=100.0)
    with sj.Context(unicomp=True) as a, sj.Context(unicomp=False) as b:
        a.sj_selfjoin_count(pts, eps)
        b.sj_selfjoin_count(pts, eps)
        ea, eb = a.sj_last_stats()["evaluations"], b.sj_last_stats()["evaluations"]
    # Without UNICOMP every ordered pair of adjacent cells (a cell with itself
    # included) costs |C_a||C_b|; with it every unordered pair of distinct
    # adjacent cells is compared once and a home cell costs |C|(|C|-1)/2.
    # Summed over cells this is exactly (full - n) / 2.
    n = 50000
    assert 2 * ea == eb - n


def test_wide_grid_uses_the_cell_frame_and_grid_frame_falls_back():
    """A range of 5e6 against eps = 1: the grid frame has no usable FP32
    margin and computes in FP64 (no rechecks); the automatic choice takes the
    cell frame and keeps the FP32 filter.  Both are exact."""
    rng = np.random.default_rng(77)
    x = np.stack([rng.uniform(0, 5e6, 20000), rng.uniform(0, 3.0, 20000)], axis=1)
    x[:200, 0] = rng.uniform(1e6, 1e6 + 20.0, 200)     # a dense stretch with many pairs
    st, _, _, _ = sj.sj_fp32_margin(2, 1.0, x.min(axis=0) - 1.0, x.max(axis=0) + 1.0)
    assert st == sj.SJ_ERANGE
    want = np.sort(orc.grid_join(x, 1.0))
    with sj.Context(frame=sj.SJ_FRAME_GRID) as ctx:
        got = np.sort(sj.pairs_to_keys(ctx.sj_selfjoin(x, 1.0)))
        stats = ctx.sj_last_stats()
        assert stats["rechecks"] == 0 and stats["frame"] == -1
    assert np.array_equal(got, want)
    with sj.Context() as ctx:
        got = np.sort(sj.pairs_to_keys(ctx.sj_selfjoin(x, 1.0)))
        assert ctx.sj_last_stats()["frame"] == sj.SJ_FRAME_CELL
        idx = ctx.sj_build_index(x, 1.0)
        info = idx.sj_index_info()
        assert info["fp32"] == 1 and info["frame"] == sj.SJ_FRAME_CELL
        idx.free()
    assert np.array_equal(got, want)


@pytest.fixture(scope="module")
def cell_ctxs():
    out = {}
    for uni in (True, False):
        for lookup in LOOKUPS:
            out[(uni, lookup)] = sj.Context(unicomp=uni, lookup=lookup, frame=sj.SJ_FRAME_CELL)
    yield out
    for c in out.values():
        c.close()


@pytest.mark.parametrize("d", [1, 2, 3, 4, 5, 6, 7, 8])
def test_cell_frame_random_all_dims(cell_ctxs, d):
    rng = np.random.default_rng(3000 + d)
    for trial in range(3):
        n = int(rng.integers(50, 3000))
        pts = rng.uniform(-10, 10, size=(n, d)) + (0.0 if trial == 0 else 1e4)
        if trial == 1:
            pts[n // 3: 2 * n // 3] = pts[: 2 * n // 3 - n // 3]   # duplicates
        k = float(rng.choice([4.0, 40.0, 400.0]))
        eps = (k * 20.0 ** d / (n * datagen.ball_volume(d))) ** (1.0 / d)
        want = orc.grid_join(pts, eps)
        for key, ctx in cell_ctxs.items():
            assert_same(gpu_keys(ctx, pts, eps), want, f"cell frame d={d} trial={trial} {key}")
            assert ctx.sj_last_stats()["frame"] == sj.SJ_FRAME_CELL


def test_cell_frame_band_pairs_and_frame_boundaries(cell_ctxs):
    """Pairs at the threshold (the FP64 recheck decides) and pairs across
    the four-cell frame boundaries, far from the origin of the grid."""
    rng = np.random.default_rng(78)
    for d in (2, 3, 6):
        eps = 0.37
        w = eps * (1.0 + 2.0 ** -16)
        base = 3e5 + rng.uniform(0, 30, size=(400, d))
        g0 = base[:, 0].min() - eps
        for p in base[::2]:
            c = int((p[0] - g0) / w)
            p[0] = g0 + (4 * (c // 4) + 4) * w - 0.5 * eps
        extra = []
        for p in base:
            v = rng.normal(size=d)
            v /= np.linalg.norm(v)
            v[0] = abs(v[0])
            f = 1.0 + float(rng.choice([-3, -1, 0, 1, 3])) * 2.0 ** -24 * float(rng.random())
            if rng.random() < 0.5:
                f = 1.0 + float(rng.integers(-4, 5)) * 2.0 ** -52
            extra.append(p + v * eps * f)
        pts = np.concatenate([base, np.array(extra)])
        want = orc.grid_join(pts, eps)
        for key, ctx in cell_ctxs.items():
            assert_same(gpu_keys(ctx, pts, eps), want, f"cell band d={d} {key}")
        ctx = cell_ctxs[(True, sj.SJ_LOOKUP_AUTO)]
        ctx.sj_selfjoin(pts, eps)
        assert ctx.sj_last_stats()["rechecks"] > 0


def test_cell_frame_config1_lattice_and_boundaries(cell_ctxs):
    cfg = datagen.CONFIG1
    pts = datagen.make_points(cfg)
    want = orc.bruteforce(pts, cfg["eps"])
    for key, ctx in cell_ctxs.items():
        assert_same(gpu_keys(ctx, pts, cfg["eps"]), want, f"cell config1 {key}")
    # unit lattice with eps = 1: 2d + 1 pairs per interior point (closed form)
    for d, m in ((2, 30), (3, 12)):
        lat = np.stack(np.meshgrid(*[np.arange(m, dtype=np.float64)] * d, indexing="ij"), -1).reshape(-1, d)
        total = m ** d + 2 * d * (m - 1) * m ** (d - 1)
        for key, ctx in cell_ctxs.items():
            assert len(ctx.sj_selfjoin(lat, 1.0)) == total, (d, key)


def wide_clusters(n, d, side, seed, sigma=0.3, per=100):
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0, side, size=(n // per, d))
    pts = centres[rng.integers(0, len(centres), n)] + rng.normal(0, sigma, size=(n, d))
    pts[: n // 20] = rng.uniform(0, side, size=(n // 20, d))       # isolated background
    return pts


@pytest.mark.parametrize("d,side,n", [(3, 1e7, 20000), (5, 1e5, 8000), (8, 1e3, 5000)])
def test_grid_of_2_63_or_more_cells(d, side, n):
    """Grids whose linear ids overflow 64 bits (about 8e21 cells at 3-D,
    1e31 at 5-D, 3e26 at 8-D) are ordered and searched by coordinate tuple;
    the result equals the definition (brute force)."""
    pts = wide_clusters(n, d, side, seed=90 + d)
    eps = 0.5
    want = orc.bruteforce(pts, eps)
    for prec in (sj.SJ_PREC_FP32_RECHECK, sj.SJ_PREC_FP64):
        for uni in (True, False):
            with sj.Context(prec=prec, unicomp=uni) as ctx:
                assert_same(gpu_keys(ctx, pts, eps), want, f"huge grid d={d} prec={prec} uni={uni}")
                if prec == sj.SJ_PREC_FP32_RECHECK:
                    assert ctx.sj_last_stats()["frame"] == sj.SJ_FRAME_CELL
                idx = ctx.sj_build_index(pts, eps)
                info = idx.sj_index_info()
                assert info["grid_cells"] == 2 ** 64 - 1 and info["dense"] == 0
                B, G, A, M = idx.sj_index_export()
                assert B is None and G[-1] == n and np.array_equal(np.sort(A), np.arange(n))
                idx.free()
    assert len(want) > n          # some pairs beyond the self-pairs


def test_coordinate_order_matches_linear_order():
    """On an ordinary grid the coordinate-tuple order is the linear-id
    order: the same A and G as the sort by linear id, and no B."""
    pts = datagen.uniform(30000, 4, seed=91)
    eps = datagen.eps_for_neighbors(30000, 4, 20)
    with sj.Context(lookup=sj.SJ_LOOKUP_SEARCH) as c1, sj.Context(lookup=sj.SJ_LOOKUP_COORDS) as c2:
        i1, i2 = c1.sj_build_index(pts, eps), c2.sj_build_index(pts, eps)
        B1, G1, A1, M1 = i1.sj_index_export()
        B2, G2, A2, M2 = i2.sj_index_export()
        assert B2 is None and B1 is not None
        assert np.array_equal(G1, G2) and np.array_equal(A1, A2) and np.array_equal(M1, M2)
        i1.free()
        i2.free()
