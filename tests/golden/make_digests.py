"""Writes the full-size expected digests of the large workloads.

Run from the repository root:  python -m tests.golden.make_digests [names]

For each workload it generates the seeded points (the input generator only
draws numbers), runs the CPU oracle's grid join (``oracle.grid_digest``:
Algorithm 1's search with the exact FP64 predicate of Section III) and
stores, in ``digests.json`` beside this file:

  * the point set's SHA-256 (so a reader can tell that the same input was
    regenerated) and epsilon as a hex float;
  * the member count, the SHA-256 of the per-point degree array (uint32,
    little-endian) and the order-independent pair hash
    sum of mix64(i << 32 | j) mod 2^64 (splitmix64 finaliser).

Nothing here touches the CUDA library: every stored value comes from the
oracle.  Workloads: the 2,000,000-point uniform sets (d = 2..6, 64 mean
neighbours), the 10,000,000-point uniform sets (d = 2..6, 128 mean
neighbours) and the 5,000,000-point clustered sets (d = 2, 3, eps = 0.5).
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import oracle as orc                       # noqa: E402
from paper_1803_04120_gb300 import datagen            # noqa: E402

PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "digests.json")


def workloads():
    out = [datagen.config2(d) for d in range(2, 7)]
    out += [datagen.config3(d) for d in range(2, 7)]
    out += [datagen.config4(d) for d in (2, 3)]
    return out


def sha256(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def digest(cfg: dict) -> dict:
    pts = datagen.make_points(cfg)
    t0 = time.time()
    count, deg, h = orc.grid_digest(pts, cfg["eps"])
    return dict(name=cfg["name"], n=cfg["n"], d=cfg["d"], seed=cfg["seed"],
                eps_hex=float(cfg["eps"]).hex(), points_sha256=sha256(pts),
                count=int(count), pair_hash=int(h),
                degree_sha256=sha256(deg.astype("<u4")),
                max_degree=int(deg.max()),
                oracle_seconds=round(time.time() - t0, 1),
                oracle_threads=orc.default_threads())


def load() -> dict:
    if os.path.exists(PATH):
        with open(PATH) as f:
            return json.load(f)
    return {}


def main(names):
    table = load()
    for cfg in workloads():
        if names and cfg["name"] not in names:
            continue
        rec = digest(cfg)
        table[cfg["name"]] = rec
        with open(PATH + ".tmp", "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
        os.replace(PATH + ".tmp", PATH)
        print(json.dumps(rec), flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
