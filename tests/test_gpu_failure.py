"""Failure detection without a GPU fault: a bounded device wait that runs
out ends the call with SJ_ETIMEOUT and leaves the context usable.

The search kernel's warps wait on mbarriers for their staged candidate
copies, each wait bounded by sj_config.wait_ms.  The context's test hook
(test_stall) makes one warp skip issuing its first copy, so nothing will
ever complete that wait and no copy is in flight for it: the wait runs out,
the warp records the time-out, waits (bounded) for its other copies and
leaves, and the host turns the error word into SJ_ETIMEOUT.  Afterwards the
same process runs joins that equal the oracle."""
import time

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1803_04120_gb300 import datagen, sj

pytestmark = pytest.mark.gpu


def test_expired_wait_returns_timeout_and_context_stays_usable():
    torch = pytest.importorskip("torch")
    pts_np = datagen.uniform(200000, 3, seed=51)
    eps = datagen.eps_for_neighbors(200000, 3, 32)
    want = orc.grid_join(pts_np, eps)
    pts = torch.from_numpy(pts_np).cuda()
    out = torch.empty((want.size + 16, 2), dtype=torch.int32, device="cuda")
    with sj.Context(autotune=False, wait_ms=200, test_stall=True) as bad:
        for _ in range(2):                       # the barriers start afresh each launch
            t0 = time.time()
            with pytest.raises(sj.SJError) as ei:
                bad.sj_selfjoin_device(pts, eps, out)
            assert ei.value.status == sj.SJ_ETIMEOUT
            assert time.time() - t0 < 30.0
        with pytest.raises(sj.SJError) as ei:    # host-result path (sampled count first)
            bad.sj_selfjoin(pts_np, eps)
        assert ei.value.status == sj.SJ_ETIMEOUT
        torch.cuda.synchronize()
    with sj.Context(autotune=False, wait_ms=200) as good:
        n = good.sj_selfjoin_device(pts, eps, out)
        assert n == want.size
        assert np.array_equal(sj.pairs_to_keys(out[:n].cpu().numpy().view(np.uint32)), want)
        assert np.array_equal(sj.pairs_to_keys(good.sj_selfjoin(pts_np, eps)), want)
