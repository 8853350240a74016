"""Full-size parity: every result pair of the large workloads, reduced to
count, per-point degree and order-independent pair hash, equals the
oracle's digest (Algorithm 1's grid search with the exact FP64 predicate of
Section III).

The oracle's digests of these workloads take minutes of CPU time, so they
are stored in tests/golden/digests.json, written by
tests/golden/make_digests.py (which calls the oracle only).  Each test first
checks that it regenerated the same input (SHA-256 of the points, epsilon
bit for bit); if not, it computes the oracle digest here instead.

Workloads: 2,000,000 uniform points (d = 2..6, 64 mean neighbours; pairs in
device memory), 10,000,000 uniform points (d = 2..6, 128 mean neighbours,
about 1.3e9 pairs; result buffers capped at 2 GB so the pairs stream out in
at least six batches, Section V-A) and 5,000,000 clustered points (d = 2, 3,
eps = 0.5; 8.2e9 and 4.8e9 pairs, heavy per-cell imbalance; streamed).
"""
import json
import os

import numpy as np
import pytest

from gpu_digest import Digest, sha256
from oracle import oracle as orc
from paper_1803_04120_gb300 import datagen, sj

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "digests.json")


def expected(cfg, pts):
    """(count, degree SHA-256, pair hash) of the oracle for cfg's input."""
    table = json.load(open(GOLDEN)) if os.path.exists(GOLDEN) else {}
    g = table.get(cfg["name"])
    if g and g["points_sha256"] == sha256(pts) and float.fromhex(g["eps_hex"]) == cfg["eps"]:
        return g["count"], g["degree_sha256"], g["pair_hash"]
    count, deg, h = orc.grid_digest(pts, cfg["eps"])
    return count, sha256(deg.astype("<u4")), h


def check(dg, want, what):
    count, deg_sha, h = want
    assert dg.count == count, (what, dg.count, count)
    assert dg.hash == h, what
    assert dg.degree_sha256() == deg_sha, what


@pytest.mark.parametrize("d", [2, 3, 4, 5, 6])
def test_config2_full_size_digest(d):
    """2,000,000 uniform points, every pair in device memory."""
    torch = pytest.importorskip("torch")
    cfg = datagen.config2(d)
    pts = datagen.make_points(cfg)
    want = expected(cfg, pts)
    with sj.Context() as ctx:
        d_pts = torch.from_numpy(pts).cuda()
        cnt = ctx.sj_selfjoin_count(d_pts, cfg["eps"])
        out = torch.empty((cnt, 2), dtype=torch.int32, device="cuda")
        assert ctx.sj_selfjoin_device(d_pts, cfg["eps"], out) == cnt
    dg = Digest(cfg["n"], "cuda")
    dg.add(out)
    check(dg, want, cfg["name"])


def streamed(cfg, pts, min_batches):
    torch = pytest.importorskip("torch")
    dg = Digest(cfg["n"], "cuda")

    def cb(pairs):
        dg.add(torch.from_numpy(pairs.view(np.int32)).cuda())
        return False

    with sj.Context(out_cap_bytes=2 << 30) as ctx:
        ctx.sj_selfjoin_stream(pts, cfg["eps"], cb)
        st = ctx.sj_last_stats()
    assert st["batches"] >= min_batches
    assert st["pairs"] == dg.count
    return dg


@pytest.mark.parametrize("d", [2, 3, 4, 5, 6])
def test_config3_full_size_streamed_digest(d):
    """10,000,000 uniform points, 128 mean neighbours, device result buffers
    capped at 2 GB: the pairs stream to the host in at least six batches."""
    cfg = datagen.config3(d)
    pts = datagen.make_points(cfg)
    want = expected(cfg, pts)
    check(streamed(cfg, pts, 6), want, cfg["name"])


@pytest.mark.parametrize("d", [2, 3])
def test_config4_clustered_full_size_streamed_digest(d):
    """5,000,000 clustered points (1,000 Gaussian clusters, sigma log-uniform
    in [0.1, 5], plus 10 % uniform background), eps = 0.5."""
    cfg = datagen.config4(d)
    pts = datagen.make_points(cfg)
    want = expected(cfg, pts)
    check(streamed(cfg, pts, 3), want, cfg["name"])
