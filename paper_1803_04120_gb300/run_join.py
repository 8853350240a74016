"""Command-line driver: runs the device-resident self-join on a synthetic
workload and prints the search-and-refine kernel time.

    python -m paper_1803_04120_gb300.run_join --dims 2,6 --reps 2

Workload: 2,000,000 uniform points in [0,100]^d with epsilon for 64 mean
neighbours (``--points`` and ``--neighbours`` change it).  Each run does one
counting join (to size the output) and then ``--reps`` timed joins; with
``--no-tune`` the join-kernel launches under a profiler are therefore
numbered 0 (count), 1, 2, ... (the tuner otherwise adds its sampled launches
before the count).
"""
from __future__ import annotations

import argparse
import json

from . import datagen, sj


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--dims", default="2,3,4,5,6")
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--points", type=int, default=2_000_000)
    ap.add_argument("--neighbours", type=float, default=64.0)
    ap.add_argument("--fp64", action="store_true", help="plain FP64 join instead of FP32 + recheck")
    ap.add_argument("--no-unicomp", action="store_true")
    ap.add_argument("--no-tune", action="store_true",
                    help="fixed launch parameters (no tuner launches before the count)")
    ap.add_argument("--grab", type=int, default=-1, help="work items per cursor bump")
    args = ap.parse_args(argv)

    import torch

    prec = sj.SJ_PREC_FP64 if args.fp64 else sj.SJ_PREC_FP32_RECHECK
    for d in [int(x) for x in args.dims.split(",")]:
        seed = 2 + d
        eps = datagen.eps_for_neighbors(args.points, d, args.neighbours)
        pts = torch.from_numpy(datagen.uniform(args.points, d, seed)).cuda()
        with sj.Context(prec=prec, unicomp=not args.no_unicomp, profile=True,
                        autotune=not args.no_tune, grab=args.grab) as ctx:
            n = ctx.sj_selfjoin_count(pts, eps)
            out = torch.empty((n, 2), dtype=torch.int32, device="cuda")
            ctx.sj_profile_read()
            for _ in range(args.reps):
                assert ctx.sj_selfjoin_device(pts, eps, out) == n
            ms, launches = ctx.sj_profile_read()
            st = ctx.sj_last_stats()
        print(json.dumps(dict(d=d, eps=eps, pairs=n, kernel_ms=round(ms / max(launches, 1), 4),
                              grab=st["grab"], nbuf=st["nbuf"], wpb=st["wpb"], staging=st["staging"],
                              tuned=st["tuned"],
                              evaluations=st["evaluations"], rechecks=st["rechecks"],
                              index_ms=round(st["ms_index"], 3))))


if __name__ == "__main__":
    main()
