"""Many joins in one pass (sj_selfjoin_multi), the serving loop
(sj_submit / sj_poll) and one join split over ranks: every job's pair set
must equal the oracle's, whatever wave or shard it ran in."""
import threading

import numpy as np
import pytest

from oracle import oracle
from paper_1803_04120_gb300 import datagen, sj

pytestmark = pytest.mark.gpu


def keys(pairs):
    return np.sort(sj.pairs_to_keys(pairs))


def oracle_keys(pts, eps):
    return np.sort(oracle.grid_join(pts, eps))


def mixed_jobs(seed, count, n_lo=50, n_hi=6000):
    """Jobs of uneven n, d in 1..8 and eps for 4..40 mean neighbours."""
    rng = np.random.default_rng(seed)
    jobs = []
    for k in range(count):
        d = int(rng.integers(1, 9))
        n = int(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi))))
        pts = datagen.uniform(n, d, seed=1000 * seed + k)
        nb = float(rng.uniform(4, 40))
        eps = datagen.eps_for_neighbors(n, d, nb)
        jobs.append((pts, eps))
    return jobs


@pytest.mark.parametrize("prec,frame", [(sj.SJ_PREC_FP32_RECHECK, sj.SJ_FRAME_AUTO),
                                        (sj.SJ_PREC_FP32_RECHECK, sj.SJ_FRAME_CELL),
                                        (sj.SJ_PREC_FP64, sj.SJ_FRAME_AUTO)])
def test_multi_matches_oracle(prec, frame):
    jobs = mixed_jobs(1, 40)
    with sj.Context(prec=prec, frame=frame) as ctx:
        res = ctx.sj_selfjoin_multi(jobs)
        st = ctx.sj_last_stats()
    assert len(res) == len(jobs)
    for (pts, eps), r in zip(jobs, res):
        assert np.array_equal(keys(r), oracle_keys(pts, eps)), (pts.shape, eps)
    assert st["pairs"] == sum(len(r) for r in res)
    assert st["batches"] == 1


def test_multi_many_waves_and_large_jobs():
    # more jobs than one wave holds, some of them large
    jobs = mixed_jobs(2, 70, n_lo=20, n_hi=3000)
    jobs.append((datagen.uniform(300000, 3, seed=5), datagen.eps_for_neighbors(300000, 3, 32)))
    jobs.append((datagen.uniform(200000, 6, seed=6), datagen.eps_for_neighbors(200000, 6, 32)))
    with sj.Context() as ctx:
        res = ctx.sj_selfjoin_multi(jobs)
        assert ctx.sj_last_stats()["batches"] >= 2
        for (pts, eps), r in zip(jobs[:-2], res[:-2]):
            assert np.array_equal(keys(r), oracle_keys(pts, eps))
        for (pts, eps), r in zip(jobs[-2:], res[-2:]):
            assert np.array_equal(keys(r), oracle_keys(pts, eps))


def test_multi_overflow_rerun_and_standalone():
    # (a) a dense blob plus two far outliers: the bounding-box estimate of
    # the pair count is far too small, so the job is re-joined alone;
    # (b) a sparse 8-D set whose grid exceeds the dense table: stand-alone
    rng = np.random.default_rng(3)
    blob = np.concatenate([rng.normal(50.0, 0.3, size=(20000, 2)),
                           np.array([[0.0, 0.0], [100.0, 100.0]])])
    sparse = rng.uniform(0, 1e6, size=(3000, 8))
    jobs = [(blob, 0.05), (sparse, 1e5), (datagen.uniform(5000, 2, seed=7), 1.0)]
    with sj.Context() as ctx:
        res = ctx.sj_selfjoin_multi(jobs)
        st = ctx.sj_last_stats()
    assert st["retries"] >= 1
    for (pts, eps), r in zip(jobs, res):
        assert np.array_equal(keys(r), oracle_keys(pts, eps))


def test_multi_per_job_errors_and_device_inputs():
    torch = pytest.importorskip("torch")
    good = datagen.uniform(3000, 3, seed=8)
    bad = good.copy()
    bad[17, 1] = np.nan
    dev = torch.from_numpy(datagen.uniform(4000, 4, seed=9)).cuda()
    jobs = [(good, 3.0), (bad, 3.0), (dev, 6.0), (good, 3.0)]
    with sj.Context() as ctx:
        res = ctx.sj_selfjoin_multi(jobs, raise_errors=False)
        assert ctx.last_multi_status == [sj.SJ_OK, sj.SJ_EINVAL, sj.SJ_OK, sj.SJ_OK]
        assert res[1] is None
        assert np.array_equal(keys(res[0]), oracle_keys(good, 3.0))
        assert np.array_equal(keys(res[3]), keys(res[0]))
        assert np.array_equal(keys(res[2]), oracle_keys(dev.cpu().numpy(), 6.0))
        with pytest.raises(sj.SJError) as ei:
            ctx.sj_selfjoin_multi(jobs)
        assert ei.value.status == sj.SJ_EINVAL
        assert ctx.sj_selfjoin_multi([]) == []


@pytest.mark.parametrize("prec", [sj.SJ_PREC_FP32_RECHECK, sj.SJ_PREC_FP64])
def test_wave_tuner_times_the_wave_and_keeps_the_result(prec):
    # a wave of 2^17 points or more is tuned the first time its key is met:
    # every job equals the oracle on the tuning wave (whose result is that of
    # the last timed launch), on the next wave (the cached choice) and with
    # the tuner off (the defaults)
    jobs = mixed_jobs(5, 48, n_lo=2000, n_hi=9000)
    assert sum(p.shape[0] for p, _ in jobs) >= 1 << 17
    want = [oracle_keys(p, e) for p, e in jobs]
    sj.sj_tune_reset()
    with sj.Context(prec=prec) as ctx:
        first = ctx.sj_selfjoin_multi(jobs)
        st1 = ctx.sj_last_stats()
        again = ctx.sj_selfjoin_multi(jobs)
        st2 = ctx.sj_last_stats()
    with sj.Context(prec=prec, autotune=False) as ctx:
        fixed = ctx.sj_selfjoin_multi(jobs)
        st0 = ctx.sj_last_stats()
    assert (st1["tuned"], st2["tuned"], st0["tuned"]) == (2, 1, 0)
    assert (st0["grab"], st0["nbuf"], st0["staging"]) == (1, 0, 0)
    assert st2["grab"] in (1, 2, 4, 8) and st2["nbuf"] in (0, 2, 3, 4)
    assert st2["staging"] in (0, 256, 512, 1024)
    for w, a, b, c in zip(want, first, again, fixed):
        assert np.array_equal(keys(a), w)
        assert np.array_equal(keys(b), w)
        assert np.array_equal(keys(c), w)


def test_multi_sorted_results():
    jobs = mixed_jobs(4, 6)
    with sj.Context(sorted=True) as ctx:
        res = ctx.sj_selfjoin_multi(jobs)
    for (pts, eps), r in zip(jobs, res):
        k = sj.pairs_to_keys(r)
        assert np.all(k[1:] > k[:-1])
        assert np.array_equal(k, oracle_keys(pts, eps))


def test_serving_mix_equals_alone():
    """Requests submitted from several threads, admitted in waves on two
    lanes: each result equals the oracle's pair set and the same join run
    alone."""
    jobs = mixed_jobs(5, 48, n_lo=100, n_hi=20000)
    jobs += [(datagen.uniform(400000, 2, seed=11), datagen.eps_for_neighbors(400000, 2, 64))]
    with sj.Context(max_inflight=16, serve_mem_bytes=2 << 30) as ctx:
        tickets = [None] * len(jobs)

        def submit(lo, hi):
            for k in range(lo, hi):
                tickets[k] = ctx.sj_submit(*jobs[k])

        th = [threading.Thread(target=submit, args=(q, min(len(jobs), q + 13)))
              for q in range(0, len(jobs), 13)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        assert len(set(tickets)) == len(jobs)
        results = {}
        for k, t in enumerate(tickets):
            r = ctx.sj_poll(t, wait_ms=120000)
            assert r is not None
            pairs, (ts, ta, td) = r
            assert 0 < ts <= ta <= td
            results[k] = pairs
        info = ctx.sj_serve_stats()
        assert info["completed"] == len(jobs) and info["queued"] == 0 and info["inflight"] == 0
        assert info["graph_launches"] >= 1 and info["lanes"] == 4
        # the oracle, and the same requests alone
        for k, (pts, eps) in enumerate(jobs):
            want = oracle_keys(pts, eps)
            assert np.array_equal(keys(results[k]), want), k
            alone = ctx.sj_selfjoin(pts, eps)
            assert np.array_equal(keys(alone), want), k
        # a consumed ticket is gone
        with pytest.raises(sj.SJError) as ei:
            ctx.sj_poll(tickets[0])
        assert ei.value.status == sj.SJ_ENOTFOUND


def test_serving_admission_and_errors():
    with sj.Context(serve_mem_bytes=64 << 20, max_inflight=2) as ctx:
        big = datagen.uniform(2000000, 2, seed=12)
        with pytest.raises(sj.SJError) as ei:
            ctx.sj_submit(big, datagen.eps_for_neighbors(2000000, 2, 64))
        assert ei.value.status == sj.SJ_ENOMEM
        with pytest.raises(sj.SJError) as ei:
            ctx.sj_submit(np.zeros((0, 2)), 1.0)
        assert ei.value.status == sj.SJ_EINVAL
        # many small requests through a tight budget: all complete, correct
        jobs = mixed_jobs(6, 20, n_lo=200, n_hi=5000)
        tickets = [ctx.sj_submit(p, e) for p, e in jobs]
        for (pts, eps), t in zip(jobs, tickets):
            r = ctx.sj_poll(t, wait_ms=120000)
            assert r is not None
            assert np.array_equal(keys(r[0]), oracle_keys(pts, eps))
        info = ctx.sj_serve_stats()
        assert info["max_wave"] <= 2
        with pytest.raises(sj.SJError) as ei:
            ctx.sj_poll(987654321)
        assert ei.value.status == sj.SJ_ENOTFOUND
        # a non-finite coordinate fails that request only, at poll time
        bad = datagen.uniform(3000, 3, seed=44)
        bad[5, 2] = np.inf
        tb = ctx.sj_submit(bad, 2.0)
        tg = ctx.sj_submit(datagen.uniform(3000, 3, seed=45), 2.0)
        with pytest.raises(sj.SJError) as ei:
            ctx.sj_poll(tb, wait_ms=60000)
        assert ei.value.status == sj.SJ_EINVAL
        assert ctx.sj_poll(tg, wait_ms=60000) is not None


def test_serving_shutdown_with_pending_requests():
    ctx = sj.Context()
    for k in range(10):
        ctx.sj_submit(datagen.uniform(50000, 3, seed=20 + k), 2.0)
    ctx.close()   # cancels what is queued, waits for what runs


def test_tuner_keeps_results():
    pts = datagen.clustered(200000, 2, seed=3)
    with sj.Context(autotune=False) as c0, sj.Context(autotune=True) as c1:
        r1 = c1.sj_selfjoin(pts, 0.5)
        s1 = c1.sj_last_stats()
        assert s1["tuned"] in (1, 2)
        assert s1["grab"] >= 1
        r0 = c0.sj_selfjoin(pts, 0.5)
        assert c0.sj_last_stats()["tuned"] == 0
        assert np.array_equal(keys(r0), keys(r1))
        n = c1.sj_selfjoin_count(pts, 0.5)
        assert c1.sj_last_stats()["tuned"] == 1
        assert n == len(r0)


@pytest.mark.parametrize("world", [2, 3, 5])
def test_shards_partition_the_join(world):
    """One join split over `world` ranks (run one after another on this GPU;
    no rank waits on another): the shards are disjoint and their union is
    the oracle's pair set."""
    torch = pytest.importorskip("torch")
    cases = [(datagen.uniform(60000, 3, seed=41), 2.5),
             (datagen.clustered(80000, 2, seed=42), 0.3),
             (datagen.uniform(30000, 5, seed=43), 12.0)]
    with sj.Context() as ctx:
        for pts_np, eps in cases:
            pts = torch.from_numpy(pts_np).cuda()
            want = oracle_keys(pts_np, eps)
            parts, total = [], 0
            for r in range(world):
                cnt = ctx.sj_selfjoin_shard_device(pts, eps, r, world, None, raise_overflow=False)
                out = torch.empty((max(cnt, 1), 2), dtype=torch.int32, device="cuda")
                assert ctx.sj_selfjoin_shard_device(pts, eps, r, world, out) == cnt
                parts.append(keys(out[:cnt].cpu().numpy()))
                total += cnt
            assert total == want.size
            got = np.sort(np.concatenate(parts))
            assert np.array_equal(got, want)
        with pytest.raises(sj.SJError) as ei:
            ctx.sj_selfjoin_shard_device(pts, eps, world, world, None)
        assert ei.value.status == sj.SJ_EINVAL


def test_bruteforce_comparator_matches_oracle():
    torch = pytest.importorskip("torch")
    cases = [(datagen.make_points(datagen.CONFIG1), datagen.CONFIG1["eps"])]
    rng = np.random.default_rng(9)
    for d in range(1, 9):
        pts = rng.uniform(0, 10, size=(int(rng.integers(1, 3000)), d))
        cases.append((pts, float(rng.uniform(0.5, 3.0))))
    with sj.Context() as ctx:
        for pts, eps in cases:
            t = torch.from_numpy(np.ascontiguousarray(pts)).cuda()
            n = ctx.sj_selfjoin_bruteforce_device(t, eps, None, raise_overflow=False)
            out = torch.empty((max(n, 1), 2), dtype=torch.int32, device="cuda")
            assert ctx.sj_selfjoin_bruteforce_device(t, eps, out) == n
            assert ctx.sj_last_stats()["evaluations"] == len(pts) ** 2
            assert np.array_equal(keys(out[:n].cpu().numpy()), oracle_keys(pts, eps)), pts.shape
