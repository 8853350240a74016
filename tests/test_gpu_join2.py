"""Two-set join R ⋈ S on the GPU against the two-set oracle."""
import numpy as np
import pytest

from oracle import oracle
from paper_1803_04120_gb300 import datagen, sj

pytestmark = pytest.mark.gpu


def run(ctx, r, s, eps):
    torch = pytest.importorskip("torch")
    n = ctx.sj_join2_device(r, s, eps, None, raise_overflow=False)
    out = torch.empty((max(n, 1), 2), dtype=torch.int32, device="cuda")
    assert ctx.sj_join2_device(r, s, eps, out) == n
    return np.sort(sj.pairs_to_keys(out[:n].cpu().numpy().view(np.uint32)))


@pytest.mark.parametrize("prec,frame", [(sj.SJ_PREC_FP32_RECHECK, sj.SJ_FRAME_AUTO),
                                        (sj.SJ_PREC_FP32_RECHECK, sj.SJ_FRAME_CELL),
                                        (sj.SJ_PREC_FP64, sj.SJ_FRAME_AUTO)])
def test_join2_matches_oracle(prec, frame):
    rng = np.random.default_rng(5)
    with sj.Context(prec=prec, frame=frame) as ctx:
        for d in range(1, 9):
            r = rng.uniform(0, 20, size=(int(rng.integers(1, 3000)), d))
            s = rng.uniform(5, 30, size=(int(rng.integers(1, 3000)), d))
            eps = float(rng.uniform(0.5, 6.0))
            assert np.array_equal(run(ctx, r, s, eps), oracle.bruteforce2(r, s, eps)), d


def test_join2_special_cases():
    rng = np.random.default_rng(6)
    with sj.Context() as ctx:
        r = datagen.uniform(4000, 3, seed=61)
        # R ⋈ R is the self-join
        assert np.array_equal(run(ctx, r, r, 4.0), np.sort(oracle.grid_join(r, 4.0)))
        # disjoint boxes: no pairs
        far = r + 1000.0
        assert len(run(ctx, r, far, 4.0)) == 0
        # one point against many, sizes 1 x n and n x 1
        one = r[:1]
        assert np.array_equal(run(ctx, one, r, 10.0), oracle.bruteforce2(one, r, 10.0))
        assert np.array_equal(run(ctx, r, one, 10.0), oracle.bruteforce2(r, one, 10.0))
        # a dense cluster against uniform background (heavy query cells)
        blob = rng.normal(50.0, 0.5, size=(5000, 2))
        bg = datagen.uniform(5000, 2, seed=62)
        assert np.array_equal(run(ctx, blob, bg, 1.0), oracle.bruteforce2(blob, bg, 1.0))
        # errors: dimensions differ, non-finite input
        with pytest.raises(ValueError):
            ctx.sj_join2_device(r, bg, 1.0, None)
        bad = r.copy()
        bad[3, 1] = np.nan
        with pytest.raises(sj.SJError) as ei:
            ctx.sj_join2_device(r, bad, 1.0, None)
        assert ei.value.status == sj.SJ_EINVAL


def test_join2_device_inputs_and_overflow():
    torch = pytest.importorskip("torch")
    r = torch.from_numpy(datagen.uniform(20000, 4, seed=63)).cuda()
    s = torch.from_numpy(datagen.uniform(30000, 4, seed=64)).cuda()
    with sj.Context() as ctx:
        n = ctx.sj_join2_device(r, s, 8.0, None, raise_overflow=False)
        small = torch.empty((10, 2), dtype=torch.int32, device="cuda")
        assert ctx.sj_join2_device(r, s, 8.0, small, raise_overflow=False) == n
        got = run(ctx, r, s, 8.0)
    assert np.array_equal(got, oracle.bruteforce2(r.cpu().numpy(), s.cpu().numpy(), 8.0))


def test_join2_on_a_grid_of_2_63_or_more_cells():
    """R and S spread over [0, 1e7]^3 with eps = 0.5: the union grid has
    about 8e21 cells and is searched by coordinate tuple."""
    rng = np.random.default_rng(65)
    centres = rng.uniform(0, 1e7, size=(60, 3))
    r = centres[rng.integers(0, 60, 3000)] + rng.normal(0, 0.3, size=(3000, 3))
    s = centres[rng.integers(0, 60, 4000)] + rng.normal(0, 0.3, size=(4000, 3))
    for prec in (sj.SJ_PREC_FP32_RECHECK, sj.SJ_PREC_FP64):
        with sj.Context(prec=prec) as ctx:
            got = run(ctx, r, s, 0.5)
        want = oracle.bruteforce2(r, s, 0.5)
        assert len(want) > 0 and np.array_equal(got, want), prec
