"""The join entry point for callers that cannot allocate memory.

sj_selfjoin_noalloc serves code that may not call cudaMalloc (for example a
plug-in running inside another framework's fixed memory budget): it takes
all working memory from the library's fixed static region.  Its pairs must
equal the CPU oracle's and those of the regular device-resident entry
point.  Each case runs twice in a row, since the region keeps the previous
call's contents.  One case has coordinates so large that no FP32 margin is
usable, so the FP64 records are carved from the region too.  This file is
collected last so that a run stopping at the first failure has already run
every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1803_04120_gb300 import datagen, sj

pytestmark = pytest.mark.gpu


def keys(out, n):
    return sj.pairs_to_keys(out[:n].cpu().numpy().view(np.uint32))


def test_noalloc_matches_oracle_and_regular_entry_point_twice():
    torch = pytest.importorskip("torch")
    cases = [
        (datagen.uniform(40000, 2, seed=31), 0.35, 0),      # many pairs per point
        (datagen.uniform(30000, 5, seed=32), 9.0, 0),       # 5-D, FP32 path with rechecks
        (datagen.uniform(40000, 2, seed=31), 0.35, 0),      # repeat of the first case
        # coordinates up to 1e19: the FP32 sums would overflow, the join
        # computes in FP64
        (datagen.uniform(20000, 3, seed=34) * 1e17, 5e17, -1),
    ]
    with sj.Context() as ctx:
        for pts_np, eps, frame in cases:
            want = orc.grid_join(pts_np, eps)
            pts = torch.from_numpy(pts_np).cuda()
            n_ref = ctx.sj_selfjoin_count(pts, eps)
            ref = torch.empty((n_ref, 2), dtype=torch.int32, device="cuda")
            assert ctx.sj_selfjoin_device(pts, eps, ref) == n_ref
            if frame < 0:
                assert ctx.sj_last_stats()["frame"] == -1      # FP64 arithmetic
            assert np.array_equal(keys(ref, n_ref), want)
            out = torch.full((n_ref + 16, 2), -1, dtype=torch.int32, device="cuda")
            for _ in range(2):
                n = sj.sj_selfjoin_noalloc(pts, eps, out)
                assert n == n_ref == want.size
                assert np.array_equal(keys(out, n), want)


def test_noalloc_limits_and_errors():
    torch = pytest.importorskip("torch")
    big = torch.zeros((70000, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(sj.SJError) as ei:
        sj.sj_selfjoin_noalloc(big, 1.0, None)
    assert ei.value.status == sj.SJ_ERANGE
    host = np.zeros((10, 2))
    with pytest.raises(sj.SJError) as ei:
        sj.sj_selfjoin_noalloc(host, 1.0, None)
    assert ei.value.status == sj.SJ_EINVAL
    # a buffer that is too small still reports the count
    pts_np = datagen.uniform(5000, 3, seed=33)
    pts = torch.from_numpy(pts_np).cuda()
    small = torch.empty((10, 2), dtype=torch.int32, device="cuda")
    n = sj.sj_selfjoin_noalloc(pts, 4.0, small, raise_overflow=False)
    assert n == orc.grid_join(pts_np, 4.0).size
