"""Throughput benchmark of the GB300 epsilon self-join.

One step = the full hot path (index build, adjacent-cell search, refine,
pair output) over the 2,000,000-point uniform workload in every dimension
d = 2..6 with epsilon set for 64 mean neighbours: five self-joins, about
5.9e8 result pairs, every pair written to device memory.

Printed JSON line (rank 0):
  value        result pairs/s of the FP32-filter + FP64-recheck join, inputs
               resident in HBM, device time of the timed steps (CUDA events
               on the launching stream; L2 flushed between steps)
  e2e          the same metric through sj_selfjoin with host input and host
               result (host->device copy of the points and device->host copy
               of every pair inside the timed region)
  fp64         the plain FP64 GPU join on the same inputs (same metric)
  roofline     the search-and-refine kernel of the dominant launch against
               max(FLOPs / FP32 peak, bytes / HBM bandwidth), the FP32 peak
               measured by the library's FMA-chain kernel in this run
  cpu_baseline the CPU oracle on the host cores: a fixed query sample per d,
               grid build timed apart, extrapolated to the whole job
  streamed_10M 10,000,000 uniform points, d = 2..6, 128 neighbours, result
               buffers capped at 2 GB: pairs streamed to pinned host memory
  skew         clustered 5,000,000 points (d = 2, 3, eps = 0.5): device join
               with the tuned launch parameters against the fixed defaults
  ablation     the join kernel with and without UNICOMP, and the indexed
               join against the index-free brute-force comparator
  serving      10,000 join requests (n log-uniform in [1e3, 1e6], d in
               2..6, 8..128 mean neighbours) through sj_submit/sj_poll, all
               at once (saturated) and with Poisson arrivals swept over
               0.25..1 of the saturated rate: p50/p99 latency and pairs/s,
               against requests joined one at a time through sj_selfjoin
  frames       FP32 record frames: grid against four-cell frame
  highdim      16-dimensional joins (uniform and clustered), FP32 against FP64
  multi        64 joins of the serving mix in one sj_selfjoin_multi call
               against the same joins one at a time
--impl reference times the CPU oracle alone (the reference arm).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1803_04120_gb300 import datagen  # noqa: E402

DIMS = (2, 3, 4, 5, 6)
METRIC = "result pairs/s FP32+FP64-recheck vs plain FP64 (exact set); serving p50/p99 ms"
UNIT = "pairs/s"
WORKLOAD = "uniform 2,000,000 points in [0,100]^d for d=2..6, eps for 64 mean neighbours"


def profiled_traffic(d: int):
    """DRAM bytes per launch of the d-dimensional join kernel from the ncu
    summary in profiles/, or None when the kernel source has changed since
    that capture (or d was not captured)."""
    import hashlib
    import re
    summ = os.path.join(ROOT, "profiles", "join_kernel_uniform2M.md")
    src = os.path.join(ROOT, "paper_1803_04120_gb300", "csrc", "join.cu")
    try:
        text = open(summ).read()
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()
    except OSError:
        return None
    m = re.search(r"kernel_source_sha256:\s*([0-9a-f]{64})", text)
    t = re.search(r"traffic_bytes_per_launch\[d=%d\]:\s*(\d+)" % d, text)
    if not m or not t or m.group(1) != h:
        return None
    return int(t.group(1))


DATA = "synthetic (seeded uniform, stands in for the paper's Syn- datasets)"


def bench_config(data):
    """The workload description both arms print (identical dicts)."""
    return {"workload": WORKLOAD, "n": 2_000_000, "dims": list(DIMS),
            "eps": [round(c["eps"], 6) for c, _ in data],
            "l2": "GPU arm: flushed between timed steps (512 MiB write); CPU arm: n/a"}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    hbm, src = 6800.0, "fallback"
    sm_mhz = 2070.0
    if os.path.exists(path):
        try:
            j = json.load(open(path))
            hbm = float(j.get("hbm_gbs", hbm))
            sm_mhz = float(j.get("sm_max_mhz", sm_mhz))
            src = "measured"
        except Exception:
            pass
    # FP32 (CUDA-core) peak: 152 SMs x 128 FP32 lanes x 2 flops x max SM clock
    fp32_tflops = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
    return hbm, src, fp32_tflops


def fp32_rate(dev: int):
    """FP32 fused multiply-add rate of the GPU (library kernel, CUDA events),
    scalar fma.rn.f32 and packed fma.rn.f32x2, with the SM clocks sampled
    meanwhile; None when the measurement fails."""
    from paper_1803_04120_gb300 import sj
    clk = ClockSampler(dev)
    clk.start()
    try:
        sc, sc_ms = sj.sj_fp32_fma_rate(dev, packed=False)
        pk, pk_ms = sj.sj_fp32_fma_rate(dev, packed=True)
    except Exception:
        clk.stop()
        return None
    c = clk.stop()
    return {"scalar_tflops": round(sc, 2), "packed_tflops": round(pk, 2),
            "packed_over_scalar": round(pk / sc, 3), "scalar_ms": round(sc_ms, 3),
            "packed_ms": round(pk_ms, 3), "sm_mhz": c.get("sm_mhz"), "reasons": c.get("reasons")}


def fp64_rate(dev: int):
    """FP64 fused multiply-add rate of the GPU (library kernel, CUDA events),
    the denominator of the plain FP64 join's roofline; None on failure."""
    from paper_1803_04120_gb300 import sj
    try:
        tf, ms = sj.sj_fp64_fma_rate(dev)
    except Exception:
        return None
    return {"tflops": round(tf, 3), "ms": round(ms, 3)}


class ClockSampler:
    """nvidia-smi samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        fd, self.path = tempfile.mkstemp(prefix="sj_clocks_", suffix=".csv")
        os.close(fd)

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        try:
            os.remove(self.path)
        except OSError:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def workload():
    out = []
    for d in DIMS:
        cfg = datagen.config2(d)
        out.append((cfg, datagen.make_points(cfg)))
    return out


# ---------------------------------------------------------------- CPU oracle

# Query points per dimension of the oracle's timed sample (the same in the
# reference arm and in the GPU arm's cpu_baseline): about a second of
# search on 16 cores each, with the grid build timed apart.
ORACLE_SAMPLE = {2: 400_000, 3: 200_000, 4: 80_000, 5: 30_000, 6: 16_000}


def oracle_build_seconds(data):
    """Grid build time of the oracle per dataset: a search pass with a
    single query is the build alone."""
    from oracle import oracle as orc
    out = {}
    for cfg, pts in data:
        t0 = time.perf_counter()
        orc.grid_neighbor_counts(pts, cfg["eps"], np.zeros(1, dtype=np.uint32))
        out[cfg["d"]] = time.perf_counter() - t0
    return out


def oracle_sample(data, build_s):
    """One timed pass of the CPU oracle (Algorithm 1's grid search, exact FP64
    predicate, all host cores) over a fixed query sample of every dataset.
    Each pass builds the grid and searches the sample; the query phase is
    the pass minus the build time.  The whole-job rate extrapolates every
    dataset to all of its points: sum of pairs x n/m over sum of
    (build + query time x n/m)."""
    from oracle import oracle as orc
    cores = orc.default_threads()
    job_pairs = job_time = q_pairs = q_time = 0.0
    for cfg, pts in data:
        n, d = pts.shape
        m = min(n, ORACLE_SAMPLE[d])
        q = np.sort(np.random.default_rng(100 + d).choice(n, size=m, replace=False)).astype(np.uint32)
        t0 = time.perf_counter()
        offs = orc.grid_neighbor_counts(pts, cfg["eps"], q, nthreads=cores)
        tq = max(time.perf_counter() - t0 - build_s[d], 1e-6)
        pairs = float(offs[-1])
        q_pairs += pairs
        q_time += tq
        job_pairs += pairs * n / m
        job_time += build_s[d] + tq * n / m
    sample = ("fixed query sample per d (" +
              ", ".join(f"d={cfg['d']}: {min(p.shape[0], ORACLE_SAMPLE[cfg['d']]):,}" for cfg, p in data) +
              " of 2,000,000 points); grid build timed apart; value extrapolates each d to all points")
    return {"value": job_pairs / job_time, "query_pairs_per_s": q_pairs / q_time,
            "build_s": {str(d): round(t, 3) for d, t in build_s.items()},
            "cores": cores, "sample": sample, "pass_s": q_time + sum(build_s.values())}


# ---------------------------------------------------------------- skew

def skew_bench(dev: int, reps: int):
    """Clustered 5,000,000-point workload (d = 2, 3, eps = 0.5), pairs in
    device memory: tuned launch parameters against the fixed defaults."""
    import torch
    from paper_1803_04120_gb300 import sj

    stream = torch.cuda.Stream()
    out = []
    for d in (2, 3):
        cfg = datagen.config4(d)
        pts = torch.from_numpy(datagen.make_points(cfg)).cuda()
        c0 = sj.Context(autotune=False, profile=True, device=dev)
        c1 = sj.Context(autotune=True, profile=True, device=dev)
        cnt = c0.sj_selfjoin_count(pts, cfg["eps"])
        buf = torch.empty((cnt, 2), dtype=torch.int32, device="cuda")
        res = {}
        for name, c in (("default", c0), ("tuned", c1)):
            c.sj_selfjoin_device(pts, cfg["eps"], buf, stream=stream)   # warm-up (tunes c1)
            torch.cuda.synchronize()
            c.sj_profile_read()
            ts = []
            for _ in range(reps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                n = c.sj_selfjoin_device(pts, cfg["eps"], buf, stream=stream)
                e1.record(stream)
                torch.cuda.synchronize()
                assert n == cnt
                ts.append(e0.elapsed_time(e1))
            kms, nl = c.sj_profile_read()
            st = c.sj_last_stats()
            res[name] = dict(ms=round(statistics.mean(ts), 3), kernel_ms=round(kms / max(nl, 1), 3),
                             grab=st["grab"], nbuf=st["nbuf"], wpb=st["wpb"], staging=st["staging"],
                             tuned=st["tuned"])
        out.append(dict(d=d, n=cfg["n"], eps=cfg["eps"], pairs=cnt,
                        default=res["default"], tuned=res["tuned"],
                        pairs_per_s_tuned=round(cnt / (res["tuned"]["ms"] / 1e3), 1),
                        speedup=round(res["default"]["ms"] / res["tuned"]["ms"], 3)))
        del buf, pts
        c0.close()
        c1.close()
        torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------- ablation

def ablation_bench(dev: int, reps: int):
    """What the index and UNICOMP save: the join kernel with and without
    UNICOMP on the 2,000,000-point workload, and the indexed join against
    the index-free brute-force comparator on config 1 and on 100,000-point
    uniform sets."""
    import torch
    from paper_1803_04120_gb300 import sj

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return min(ts)

    uni = []
    for d in DIMS:
        cfg = datagen.config2(d)
        pts = torch.from_numpy(datagen.make_points(cfg)).cuda()
        row = {"d": d}
        for flag in (1, 0):
            with sj.Context(unicomp=bool(flag), profile=True, device=dev) as c:
                n = c.sj_selfjoin_count(pts, cfg["eps"])
                out = torch.empty((n, 2), dtype=torch.int32, device="cuda")
                c.sj_selfjoin_device(pts, cfg["eps"], out)
                c.sj_profile_read()
                for _ in range(reps):
                    c.sj_selfjoin_device(pts, cfg["eps"], out)
                ms, nl = c.sj_profile_read()
                st = c.sj_last_stats()
                key = "unicomp" if flag else "full_search"
                row[key] = {"kernel_ms": round(ms / max(nl, 1), 3), "evaluations": st["evaluations"]}
                del out
        row["time_ratio"] = round(row["full_search"]["kernel_ms"] / row["unicomp"]["kernel_ms"], 3)
        row["evaluation_ratio"] = round(row["full_search"]["evaluations"] / row["unicomp"]["evaluations"], 3)
        uni.append(row)
    brute = []
    cases = [("config 1: 20,000 points, d=2, eps=2", datagen.make_points(datagen.CONFIG1),
              datagen.CONFIG1["eps"])]
    for d in (2, 4, 6):
        cases.append((f"100,000 uniform points, d={d}, 64 neighbours", datagen.uniform(100000, d, 70 + d),
                      datagen.eps_for_neighbors(100000, d, 64)))
    with sj.Context(device=dev) as c:
        for name, pts_np, eps in cases:
            pts = torch.from_numpy(pts_np).cuda()
            n = c.sj_selfjoin_count(pts, eps)
            out = torch.empty((n, 2), dtype=torch.int32, device="cuda")
            t_idx = timed(lambda: c.sj_selfjoin_device(pts, eps, out))
            t_bf = timed(lambda: c.sj_selfjoin_bruteforce_device(pts, eps, out))
            brute.append({"workload": name, "pairs": n, "indexed_ms": round(t_idx, 3),
                          "bruteforce_ms": round(t_bf, 3), "speedup": round(t_bf / t_idx, 1)})
    return {"unicomp_vs_full_search": uni, "index_vs_bruteforce": brute,
            "note": "join kernel only for UNICOMP; whole device call (index build included) "
                    "for the brute-force comparison"}


# ---------------------------------------------------------------- record frames

def frame_bench(dev: int, reps: int):
    """FP32 record frames.  Wide-domain clustered points (2,000,000 points,
    about 2e6 cells per dimension): records relative to g_min leave no
    usable FP32 margin there and the join computes in FP64, records relative
    to the four-cell frame keep the FP32 filter.  On the 2,000,000-point
    uniform workload (d = 2, 6): the cost of the frame step against the
    rechecks it saves.  Pairs in device memory; whole call (index build
    included) and join kernel times."""
    import torch
    from paper_1803_04120_gb300 import sj

    stream = torch.cuda.Stream()

    def measure(cfg, frame):
        pts = torch.from_numpy(datagen.make_points(cfg)).cuda()
        with sj.Context(frame=frame, profile=True, device=dev) as c:
            n = c.sj_selfjoin_count(pts, cfg["eps"])
            out = torch.empty((max(n, 1), 2), dtype=torch.int32, device="cuda")
            c.sj_selfjoin_device(pts, cfg["eps"], out, stream=stream)
            torch.cuda.synchronize()
            c.sj_profile_read()
            ts = []
            for _ in range(reps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                assert c.sj_selfjoin_device(pts, cfg["eps"], out, stream=stream) == n
                e1.record(stream)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            kms, nl = c.sj_profile_read()
            st = c.sj_last_stats()
        del out, pts
        torch.cuda.empty_cache()
        return n, {"ms": round(min(ts), 3), "kernel_ms": round(kms / max(nl, 1), 3),
                   "rechecks": st["rechecks"],
                   "arithmetic": {-1: "fp64", 0: "fp32 grid frame", 1: "fp32 cell frame"}[st["frame"]]}

    wide = []
    for d in (2, 3):
        cfg = datagen.wide_clustered(d)
        n, auto = measure(cfg, sj.SJ_FRAME_AUTO)
        _, grid = measure(cfg, sj.SJ_FRAME_GRID)
        wide.append({"d": d, "n": cfg["n"], "eps": cfg["eps"], "pairs": n,
                     "auto": auto, "grid_frame_only": grid,
                     "pairs_per_s_auto": round(n / (auto["ms"] / 1e3), 1),
                     "speedup": round(grid["ms"] / auto["ms"], 2)})
    uni = []
    for d in (2, 6):
        cfg = datagen.config2(d)
        n, grid = measure(cfg, sj.SJ_FRAME_GRID)
        _, cell = measure(cfg, sj.SJ_FRAME_CELL)
        uni.append({"d": d, "pairs": n, "grid": grid, "cell": cell,
                    "kernel_ratio_cell_over_grid": round(cell["kernel_ms"] / grid["kernel_ms"], 3)})
    return {"wide_clustered": wide, "uniform_2M": uni,
            "workload": "wide: 2,000,000 points, 20,000 Gaussian clusters (sigma log-U[0.1, 5]) "
                        "with centres U[0, 1e6]^d plus 10% uniform background, eps = 0.5"}


# ---------------------------------------------------------------- more than 8 dimensions

def highdim_bench(dev: int, reps: int):
    """Points of 16 dimensions (grid over the six with the most cells, the
    FP32 filter over all sixteen: expanded form for the uniform set,
    difference form for the clustered one): uniform and clustered
    workloads, the FP32 filter with FP64 recheck against plain FP64, pairs
    in device memory, whole call (index build included)."""
    import torch
    from paper_1803_04120_gb300 import sj

    rng = np.random.default_rng(16)
    d = 16
    n_u = 200_000
    eps_u = (64.0 * 100.0 ** d / (n_u * datagen.ball_volume(d))) ** (1.0 / d)
    uni = datagen.uniform(n_u, d, seed=161)
    n_c = 1_000_000
    centres = rng.uniform(0, 100, size=(1000, d))
    clu = centres[rng.integers(0, 1000, n_c)] + rng.normal(0, 2.0, size=(n_c, d))
    cases = [(f"uniform {n_u:,} points in [0,100]^16, 64 neighbours", uni, eps_u),
             (f"{n_c:,} points in 1,000 Gaussian clusters (sigma 2) in [0,100]^16", clu, 8.0)]
    stream = torch.cuda.Stream()
    out = []
    for name, pts_np, eps in cases:
        pts = torch.from_numpy(pts_np).cuda()
        row = {"workload": name, "n": len(pts_np), "d": d, "eps": round(eps, 4)}
        for key, prec in (("fp32", sj.SJ_PREC_FP32_RECHECK), ("fp64", sj.SJ_PREC_FP64)):
            with sj.Context(prec=prec, profile=True, device=dev) as c:
                n = c.sj_selfjoin_count(pts, eps)
                buf = torch.empty((max(n, 1), 2), dtype=torch.int32, device="cuda")
                c.sj_selfjoin_device(pts, eps, buf, stream=stream)
                torch.cuda.synchronize()
                c.sj_profile_read()
                ts = []
                for _ in range(reps if prec == sj.SJ_PREC_FP32_RECHECK else 1):
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    assert c.sj_selfjoin_device(pts, eps, buf, stream=stream) == n
                    e1.record(stream)
                    torch.cuda.synchronize()
                    ts.append(e0.elapsed_time(e1))
                kms, nl = c.sj_profile_read()
                st = c.sj_last_stats()
                del buf
            row["pairs"] = n
            row[key] = {"ms": round(min(ts), 3), "kernel_ms": round(kms / max(nl, 1), 3),
                        "evaluations": st["evaluations"], "rechecks": st["rechecks"],
                        "pairs_per_s": round(n / (min(ts) / 1e3), 1),
                        "evaluations_per_s": round(st["evaluations"] / (kms / max(nl, 1) / 1e3), 1)}
        row["speedup_fp32"] = round(row["fp64"]["ms"] / row["fp32"]["ms"], 2)
        out.append(row)
        del pts
        torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------- serving

def _pct(v, q):
    return round(float(np.percentile(np.asarray(v) * 1e3, q)), 3)


SWEEP = (0.25, 0.5, 0.75, 1.0)


def serving_bench(dev: int, n_req: int, seed: int = 5, baseline_req: int = 500):
    """The request stream of n_req self-joins through the serving loop:
    all at once (saturated), then Poisson arrivals swept over fractions of
    the saturated request rate; against one-at-a-time joins of the first
    baseline_req requests through sj_selfjoin (plain FP64 and FP32).
    Request r takes the first n_r points of one of four pooled uniform sets
    of its dimension (10,000 independent sets of up to 1e6 points would not
    fit in host memory); every request is joined in full."""
    import threading
    from paper_1803_04120_gb300 import sj

    reqs = datagen.serving_requests(n_req, seed, rate_hz=1.0)
    pools = {d: [datagen.uniform(1_000_000, d, seed=9000 + 10 * d + k) for k in range(4)]
             for d in range(2, 7)}
    pts = [pools[r["d"]][k % 4][: r["n"]] for k, r in enumerate(reqs)]
    nb = min(baseline_req, n_req)

    def one_at_a_time(prec):
        with sj.Context(prec=prec, device=dev) as c:
            r = c.sj_selfjoin_raw(pts[0], reqs[0]["eps"])
            c.sj_result_free(r)
            lat, tot = [], 0
            t0 = time.perf_counter()
            for p, q in zip(pts[:nb], reqs[:nb]):
                t = time.perf_counter()
                r = c.sj_selfjoin_raw(p, q["eps"])
                tot += c.sj_result_count(r)
                c.sj_result_free(r)
                lat.append(time.perf_counter() - t)
            return tot, time.perf_counter() - t0, lat

    tot64, wall64, lat64 = one_at_a_time(sj.SJ_PREC_FP64)
    tot32, wall32, lat32 = one_at_a_time(sj.SJ_PREC_FP32_RECHECK)
    assert tot64 == tot32
    ctx_on = sj.Context(device=dev, max_inflight=64, serve_mem_bytes=64 << 30)
    for k in range(min(8, n_req)):        # engines, graphs, pinned buffers
        ctx_on.sj_poll(ctx_on.sj_submit(pts[k], reqs[k]["eps"]), wait_ms=60000, copy=False)

    def run(arrivals, ctx=None):
        ctx = ctx or ctx_on
        n = len(arrivals)
        tickets, got = [None] * n, [None] * n
        ready = threading.Semaphore(0)

        def poller():
            for k in range(n):
                ready.acquire()
                while got[k] is None:
                    got[k] = ctx.sj_poll(tickets[k], wait_ms=1000, copy=False)

        th = threading.Thread(target=poller)
        th.start()
        t0 = time.perf_counter()
        for k in range(n):
            dt = arrivals[k] - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            tickets[k] = ctx.sj_submit(pts[k], reqs[k]["eps"])
            ready.release()
        th.join()
        lat = [td - ts for _, (ts, ta, td) in got]
        wall = max(td for _, (ts, ta, td) in got) - min(ts for _, (ts, ta, td) in got)
        return sum(c for c, _ in got), wall, lat

    run([0.0] * nb)                       # untimed pass: pinned result buffers, pool
    run([0.0] * n_req)                    # untimed: the wave tuner meets the saturated waves' keys
    tune_info = ctx_on.sj_serve_stats()
    p_sat, wall_sat, lat_sat = run([0.0] * n_req)
    assert n_req > nb or p_sat == tot64
    rate_sat = n_req / wall_sat
    sweep = []
    for f in SWEEP:
        arrivals = [r["arrival_s"] for r in datagen.serving_requests(n_req, seed, rate_hz=f * rate_sat)]
        p_poi, wall_poi, lat_poi = run(arrivals)
        assert p_poi == p_sat
        sweep.append({"load": f, "offered_req_per_s": round(f * rate_sat, 1),
                      "req_per_s": round(n_req / wall_poi, 1),
                      "pairs_per_s": round(p_poi / wall_poi, 1),
                      "p50_ms": _pct(lat_poi, 50), "p99_ms": _pct(lat_poi, 99)})
    # the saturated stream with the wave tuner's choices and with the fixed
    # launch parameters, runs interleaved (two each)
    ctx_off = sj.Context(device=dev, max_inflight=64, serve_mem_bytes=64 << 30, autotune=False)
    run([0.0] * nb, ctx_off)
    cmp_on, cmp_off = [], []
    for _ in range(2):
        for ctx_, acc in ((ctx_off, cmp_off), (ctx_on, cmp_on)):
            p_c, wall_c, lat_c = run([0.0] * n_req, ctx_)
            assert p_c == p_sat
            acc.append({"pairs_per_s": round(p_c / wall_c, 1), "p50_ms": _pct(lat_c, 50),
                        "p99_ms": _pct(lat_c, 99)})
    ctx_off.close()
    info = ctx_on.sj_serve_stats()
    ctx_on.close()
    return {
        "requests": n_req, "pairs": p_sat,
        "request_mix": "n log-uniform [1e3,1e6], d uniform {2..6}, eps for U[8,128] mean neighbours, "
                       "uniform [0,100]^d: the first n points of one of four pooled seeded sets per d",
        "saturated": {"pairs_per_s": round(p_sat / wall_sat, 1), "req_per_s": round(rate_sat, 1),
                      "p50_ms": _pct(lat_sat, 50), "p99_ms": _pct(lat_sat, 99)},
        "sweep": sweep,
        "saturated_wave_tuner_vs_fixed_launch": {"wave_tuner": cmp_on, "fixed": cmp_off,
                                                 "order": "fixed, tuner, fixed, tuner"},
        "wave_tuner": {"tuned_waves": info["tuned_waves"], "ms_tune": round(info["ms_tune"], 1),
                       "tuned_waves_in_timed_passes": info["tuned_waves"] - tune_info["tuned_waves"]},
        "one_at_a_time_fp64": {"requests": nb, "pairs_per_s": round(tot64 / wall64, 1),
                               "p50_ms": _pct(lat64, 50), "p99_ms": _pct(lat64, 99)},
        "one_at_a_time_fp32": {"requests": nb, "pairs_per_s": round(tot32 / wall32, 1),
                               "p50_ms": _pct(lat32, 50), "p99_ms": _pct(lat32, 99)},
        "speedup_vs_plain_one_at_a_time": round((p_sat / wall_sat) / (tot64 / wall64), 2),
        "waves": info["waves"], "max_wave": info["max_wave"],
        "max_concurrent_waves": info["max_concurrent_waves"], "overflow_reruns": info["overflow_reruns"],
        "standalone": info["standalone"],
        "lane_ms": {"bounds": round(info["ms_bounds"], 1), "graph": round(info["ms_graph"], 1),
                    "output": round(info["ms_output"], 1)},
    }


# ---------------------------------------------------------------- streamed 10M

def multi_bench(dev: int, reps: int, n_jobs: int = 64, seed: int = 7):
    """Many joins in one call (sj_selfjoin_multi: one batched index build and
    one persistent multi-join launch per wave, replayed as a CUDA graph, the
    pairs delivered to host memory) against the same joins one at a time
    through sj_selfjoin (host pairs) and sj_selfjoin_device (pairs left on
    the device).  Jobs: the request mix of the serving stream (n log-uniform
    [1e3, 1e6], d uniform {2..6}, eps for U[8, 128] mean neighbours), each
    on its own seeded uniform set."""
    import torch
    from paper_1803_04120_gb300 import sj

    reqs = datagen.serving_requests(n_jobs, seed, rate_hz=1.0)
    pts = [datagen.uniform(r["n"], r["d"], seed=7000 + k) for k, r in enumerate(reqs)]
    jobs = [(p, r["eps"]) for p, r in zip(pts, reqs)]
    sj.sj_tune_reset()
    with sj.Context(device=dev) as c, sj.Context(device=dev, autotune=False) as cf:
        t0 = time.perf_counter()
        counts = c.sj_selfjoin_multi(jobs, copy=False)          # waves tuned here
        t_tuning = time.perf_counter() - t0
        assert cf.sj_selfjoin_multi(jobs, copy=False) == counts  # engines, graphs, pools
        assert c.sj_selfjoin_multi(jobs, copy=False) == counts
        total = sum(counts)
        # the wave tuner's choice and the fixed launch parameters, calls interleaved
        t_multi, t_fixed = [], []
        for _ in range(reps):
            for ctx_, t_ in ((cf, t_fixed), (c, t_multi)):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                got = ctx_.sj_selfjoin_multi(jobs, copy=False)
                t_.append(time.perf_counter() - t0)
                assert got == counts
        c.sj_selfjoin_multi(jobs, copy=False)
        lst = c.sj_last_stats()
        choice = {"tuned": lst["tuned"], "grab": lst["grab"], "nbuf": lst["nbuf"],
                  "staging": lst["staging"], "waves": lst["batches"]}
        for p, e in jobs[:4]:                                    # warm the single-join path
            c.sj_result_free(c.sj_selfjoin_raw(p, e))
        t_host = []
        for _ in range(reps):
            t0 = time.perf_counter()
            tot = 0
            for p, e in jobs:
                r = c.sj_selfjoin_raw(p, e)
                tot += c.sj_result_count(r)
                c.sj_result_free(r)
            t_host.append(time.perf_counter() - t0)
            assert tot == total
        dpts = [torch.from_numpy(p).cuda() for p in pts]
        outs = [torch.empty((max(k, 1), 2), dtype=torch.int32, device="cuda") for k in counts]
        t_dev = []
        for rep in range(reps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            tot = sum(c.sj_selfjoin_device(p, e, o) for p, (_, e), o in zip(dpts, jobs, outs))
            torch.cuda.synchronize()
            if rep:
                t_dev.append(time.perf_counter() - t0)
            assert tot == total
    ms = lambda t: round(1e3 * statistics.median(t), 3)
    return {"jobs": n_jobs, "pairs": total,
            "points": sum(int(p.shape[0]) for p in pts),
            "multi_host_pairs": {"ms": ms(t_multi), "pairs_per_s": round(total / statistics.median(t_multi), 1),
                                 "launch": "wave tuner", "last_wave_choice": choice,
                                 "tuning_call_ms": round(1e3 * t_tuning, 3)},
            "multi_host_pairs_fixed_launch": {"ms": ms(t_fixed),
                                              "pairs_per_s": round(total / statistics.median(t_fixed), 1)},
            "one_at_a_time_host_pairs": {"ms": ms(t_host),
                                         "pairs_per_s": round(total / statistics.median(t_host), 1)},
            "one_at_a_time_device_pairs": {"ms": ms(t_dev),
                                           "pairs_per_s": round(total / statistics.median(t_dev), 1)},
            "job_mix": "n log-uniform [1e3, 1e6], d uniform {2..6}, eps for U[8, 128] mean "
                       "neighbours, uniform [0, 100]^d, one seeded set per job; host inputs are "
                       "pageable numpy arrays for the host-pair rows",
            "statistic": "median of %d calls (wave-tuner and fixed-launch calls interleaved)" % reps}


def stream_bench(dev: int, reps: int):
    """10,000,000 uniform points for d = 2..6 with 128 mean neighbours (about
    1.3e9 pairs each), device result buffers capped at 2 GB: the pairs stream
    to pinned host memory in batches (Section V-A), each batch's kernel
    overlapped with the previous batch's copy.  End-to-end pairs/s (host
    points in, every pair delivered to the host), the batch count, and the
    join kernels' share of the wall time."""
    from paper_1803_04120_gb300 import sj

    out = []
    with sj.Context(device=dev, out_cap_bytes=2 << 30, profile=True) as ctx:
        for d in DIMS:
            cfg = datagen.config3(d)
            pts = datagen.make_points(cfg)
            got = [0]

            def cb(k):
                got[0] += k
                return False

            ctx.sj_selfjoin_stream(pts, cfg["eps"], cb, copy=False)    # warm-up (tunes)
            best, st, kms = None, None, 0.0
            for _ in range(reps):
                got[0] = 0
                ctx.sj_profile_read()
                t0 = time.perf_counter()
                ctx.sj_selfjoin_stream(pts, cfg["eps"], cb, copy=False)
                t = time.perf_counter() - t0
                ms, _ = ctx.sj_profile_read()
                if best is None or t < best:
                    best, st, kms = t, ctx.sj_last_stats(), ms
            pairs = got[0]
            out.append({"d": d, "n": cfg["n"], "eps": round(cfg["eps"], 6), "pairs": pairs,
                        "batches": st["batches"], "retries": st["retries"],
                        "wall_ms": round(best * 1e3, 2), "pairs_per_s": round(pairs / best, 1),
                        "join_kernels_ms": round(kms, 2),
                        "d2h_gb_per_s": round(8 * pairs / best / 1e9, 1)})
    return {"workload": "uniform 10,000,000 points in [0,100]^d, d=2..6, eps for 128 mean "
                        "neighbours, out_cap_bytes = 2 GB, sj_selfjoin_stream (host points in, "
                        "pairs to pinned host memory)", "per_d": out,
            "pairs_per_s": round(sum(r["pairs"] for r in out) / sum(r["wall_ms"] / 1e3 for r in out), 1)}


# ---------------------------------------------------------------- GPU arm

def run_gpu(args):
    import torch
    from paper_1803_04120_gb300 import sj

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    data = workload()
    stream = torch.cuda.Stream()
    d_pts = [torch.from_numpy(p).cuda() for _, p in data]
    ctx32 = [sj.Context(prec=sj.SJ_PREC_FP32_RECHECK, device=dev, profile=True) for _ in DIMS]
    ctx64 = [sj.Context(prec=sj.SJ_PREC_FP64, device=dev, profile=True) for _ in DIMS]
    counts = [c.sj_selfjoin_count(p, cfg["eps"]) for c, p, (cfg, _) in zip(ctx32, d_pts, data)]
    outs = [torch.empty((c, 2), dtype=torch.int32, device="cuda") for c in counts]
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    pairs_step = sum(counts)

    def step(ctxs, s):
        tot = 0
        for c, p, o, (cfg, _) in zip(ctxs, d_pts, outs, data):
            tot += c.sj_selfjoin_device(p, cfg["eps"], o, stream=s)
        return tot

    def timed(ctxs, steps, warmup):
        for _ in range(warmup):
            with torch.cuda.stream(stream):
                step(ctxs, stream)
        torch.cuda.synchronize()
        for c in ctxs:
            c.sj_profile_read() if c.config.profile else None
        times, launches = [], 0
        for _ in range(steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            n = step(ctxs, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            assert n == pairs_step, (n, pairs_step)
            times.append(e0.elapsed_time(e1))
            # each context made one call in the step: its last call's kernel
            # count, read after the timed region so that the calls run back
            # to back inside it
            launches += sum(c.sj_last_stats()["kernel_launches"] for c in ctxs)
        return times, launches

    clk = ClockSampler(dev)
    clk.start()
    t32, launches = timed(ctx32, args.steps, args.warmup)
    clocks = clk.stop()
    prof = [c.sj_profile_read() for c in ctx32]        # per-d join kernel (ms total, launches)
    stats = []
    for c, p, (cfg, _) in zip(ctx32, d_pts, data):     # evaluations per d (one extra count pass)
        c.sj_selfjoin_count(p, cfg["eps"])
        stats.append(c.sj_last_stats())
    ms_step = sum(t32) / len(t32)
    value = pairs_step / (ms_step / 1e3)

    # plain FP64 join, same inputs, fewer steps (it is much slower)
    t64, _ = timed(ctx64, max(1, min(args.steps, 2)), 1)
    fp64_value = pairs_step / (sum(t64) / len(t64) / 1e3)
    prof64 = [c.sj_profile_read() for c in ctx64]

    # end to end: host points in, host pairs out, through sj_selfjoin
    host_pts = [torch.from_numpy(p).pin_memory() for _, p in data]
    e2e_times = []
    for it in range(1 + 5):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tot = 0
        for c, hp, (cfg, _) in zip(ctx32, host_pts, data):
            r = c.sj_selfjoin_raw(hp.numpy(), cfg["eps"])
            tot += c.sj_result_count(r)
            c.sj_result_free(r)
        torch.cuda.synchronize()
        if it > 0:
            e2e_times.append(time.perf_counter() - t0)
        assert tot == pairs_step
    # median over five steps: a host-side stall (pinned memory, the OS) can
    # add tens of ms to one step; the mean is reported beside it
    e2e_value = pairs_step / statistics.median(e2e_times)
    e2e_mean = pairs_step / (sum(e2e_times) / len(e2e_times))
    h2d = sum(p.nbytes for _, p in data)

    # roofline of the join kernel, per launch, per d; the FP32 peak is the
    # FMA rate measured here (scalar and packed f32x2, the faster one)
    hbm, psrc, fp32_derived = peaks()
    fma = fp32_rate(dev)
    fp32 = max(fma["scalar_tflops"], fma["packed_tflops"]) if fma else fp32_derived
    roof_all = []
    for (cfg, pts), (ms, nl), st, cnt in zip(data, prof, stats, counts):
        d = cfg["d"]
        t = ms / max(nl, 1) / 1e3
        flops = (3 * d - 1) * st["evaluations"]
        byts = 8 * pts.size + 8 * cnt
        t_alu, t_hbm = flops / (fp32 * 1e12), byts / (hbm * 1e9)
        bound = "alu" if t_alu >= t_hbm else "hbm"
        if bound == "alu":
            ach, pk, unit = flops / t / 1e12, fp32, "TFLOP/s"
        else:
            ach, pk, unit = byts / t / 1e9, hbm, "GB/s"
        roof_all.append(dict(d=d, bound=bound, achieved=round(ach, 3), peak=round(pk, 1), unit=unit,
                             frac=round(ach / pk, 4), kernel_ms=round(t * 1e3, 4),
                             roofline_ms=round(max(t_alu, t_hbm) * 1e3, 4),
                             evaluations=st["evaluations"], pairs=cnt, rechecks=st["rechecks"]))
    # the plain FP64 join against the measured FP64 FMA rate: its exact
    # predicate is d subtractions, d multiplications and d - 1 additions per
    # evaluation, none fused, so it can reach at most half of the FMA rate
    f64 = fp64_rate(dev)
    roof64 = []
    for (cfg, pts), (ms, nl), st in zip(data, prof64, stats):
        d = cfg["d"]
        t = ms / max(nl, 1) / 1e3
        flops = (3 * d - 1) * st["evaluations"]
        ach = flops / t / 1e12
        roof64.append(dict(d=d, kernel_ms=round(t * 1e3, 4), achieved=round(ach, 4),
                           peak=f64["tflops"] if f64 else None, unit="TFLOP/s",
                           frac=round(ach / f64["tflops"], 4) if f64 else None))
    dom = max(roof_all, key=lambda r: r["kernel_ms"])
    roofline = dict(bound=dom["bound"], achieved=dom["achieved"], peak=dom["peak"], unit=dom["unit"],
                    frac=dom["frac"], traffic=profiled_traffic(dom["d"]),
                    traffic_source="ncu dram__bytes_read.sum + dram__bytes_write.sum, one launch "
                                   "(profiles/join_kernel_uniform2M.md); null when the kernel changed",
                    kernel=f"join_kernel d={dom['d']}",
                    peak_source=(("measured: FP32 FMA chains on every SM (sj_fp32_fma_rate), faster of "
                                  "scalar and f32x2" if fma else
                                  "derived: 152 SMs x 128 lanes x 2 x max SM clock")
                                 if dom["bound"] == "alu" else f"hbm_gbs {psrc}"),
                    all_launches_frac=round(sum(r["roofline_ms"] for r in roof_all)
                                            / sum(r["kernel_ms"] for r in roof_all), 4))

    line = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": DATA, "config": bench_config(data), "pairs_per_step": pairs_step,
        "precision": "FP32 filter with proven margin + FP64 recheck (exact set), UNICOMP",
        "fp64": {"value": round(fp64_value, 1), "unit": UNIT,
                 "ms_per_step": round(sum(t64) / len(t64), 4), "speedup_fp32": round(value / fp64_value, 2),
                 "roofline_all": roof64,
                 "peak_source": "measured: FP64 FMA chains on every SM (sj_fp64_fma_rate); "
                                "the join's unfused FP64 operations can reach at most half of it",
                 "fp64_peak": f64},
        "e2e": {"value": round(e2e_value, 1), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": 8 * pairs_step, "steps": len(e2e_times),
                "statistic": "median step time", "value_mean": round(e2e_mean, 1)},
        "gpu_launches": launches,
        "roofline": roofline,
        "roofline_all": roof_all,
        "fp32_peak": dict(fma or {}, derived_tflops=round(fp32_derived, 1)),
        "clocks": clocks,
    }
    for c in ctx32 + ctx64:
        c.close()
    del outs
    torch.cuda.empty_cache()
    if not args.no_stream:
        line["streamed_10M"] = stream_bench(dev, max(1, min(args.steps, 3)))
    if args.serve_requests > 0:
        line["serving"] = serving_bench(dev, args.serve_requests)
    if not args.no_skew:
        line["skew"] = skew_bench(dev, max(1, min(args.steps, 3)))
    if not args.no_ablation:
        line["ablation"] = ablation_bench(dev, max(1, min(args.steps, 3)))
    if not args.no_frames:
        line["frames"] = frame_bench(dev, max(1, min(args.steps, 3)))
    if not args.no_highdim:
        line["highdim"] = highdim_bench(dev, max(1, min(args.steps, 3)))
    if not args.no_multi:
        line["multi"] = multi_bench(dev, max(1, min(args.steps, 3)))
    if not args.no_cpu:
        r = oracle_sample(data, oracle_build_seconds(data))
        line["cpu_baseline"] = {"value": round(r["value"], 1), "unit": UNIT, "cores": r["cores"],
                                "kind": "oracle", "sample": r["sample"],
                                "query_pairs_per_s": round(r["query_pairs_per_s"], 1),
                                "build_s": r["build_s"]}
    return line


def replica_value(ms_local: float, pairs_per_step: int, device: str):
    """Replicas: the slowest rank's step time and the whole-job pairs/s
    (every rank processes pairs_per_step per step)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = float(t.item())
    return ms, dist.get_world_size() * pairs_per_step / (ms / 1e3)


def run_reference(args):
    """The reference arm: the CPU oracle alone, each step one timed pass over
    the fixed query sample of every dataset (oracle_sample), on all host
    cores.  Under torchrun only rank 0 runs."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    data = workload()
    build_s = oracle_build_seconds(data)
    for _ in range(args.warmup):
        oracle_sample(data, build_s)
    vals, qvals, t_all, r = [], [], [], None
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = oracle_sample(data, build_s)
        t_all.append(time.perf_counter() - t0)
        vals.append(r["value"])
        qvals.append(r["query_pairs_per_s"])
    value = statistics.mean(vals)
    return {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": 0, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(1e3 * statistics.mean(t_all), 2),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": DATA, "impl": "reference", "config": bench_config(data),
        "precision": "FP64 (the definition; the CPU oracle, Algorithm 1 without UNICOMP)",
        "cpu_baseline": {"value": round(value, 1), "unit": UNIT, "cores": r["cores"], "kind": "oracle",
                         "sample": r["sample"],
                         "query_pairs_per_s": round(statistics.mean(qvals), 1),
                         "build_s": r["build_s"]},
        "e2e": {"value": round(value, 1), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--serve-requests", type=int, default=10000,
                    help="requests of the serving stream (0: skip)")
    ap.add_argument("--no-stream", action="store_true",
                    help="skip the streamed 10,000,000-point workloads")
    ap.add_argument("--no-skew", action="store_true", help="skip the clustered workload")
    ap.add_argument("--no-ablation", action="store_true",
                    help="skip the UNICOMP and brute-force comparisons")
    ap.add_argument("--no-frames", action="store_true",
                    help="skip the FP32 record-frame comparison")
    ap.add_argument("--no-multi", action="store_true",
                    help="skip the many-joins-in-one-call comparison")
    ap.add_argument("--no-highdim", action="store_true",
                    help="skip the 16-dimensional workloads")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        line = run_reference(args)
        if line:
            print(json.dumps(line))
        return
    if world > 1:
        # replicas: each rank runs the same workload on its own GPU; the
        # whole-job value is the sum over ranks of pairs over the max time
        # (the serving and clustered sections are single-GPU measurements)
        args.serve_requests, args.no_skew, args.no_ablation, args.no_frames = 0, True, True, True
        args.no_highdim = args.no_stream = True
        import torch.distributed as dist
        dist.init_process_group("nccl")
        args.no_cpu = args.no_cpu or rank != 0
        line = run_gpu(args)
        ms, value = replica_value(line["ms_per_step"], line["config"]["pairs_per_step"], "cuda")
        if rank == 0:
            line["n_gpus"] = world
            line["ms_per_step"] = round(ms, 4)
            line["value"] = round(value, 1)
            line["config"]["parallelism"] = f"replicas x{world}"
            print(json.dumps(line))
        dist.destroy_process_group()
        return
    print(json.dumps(run_gpu(args)))


if __name__ == "__main__":
    main()
