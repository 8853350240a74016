"""Host logic of the multi-rank paths, on the CPU: the shard rule of
sj_selfjoin_shard_device (ranges of work items cut at cell starts) and the
replica aggregation of bench.py, with world_size 2 gloo process groups."""
import os
import socket

import numpy as np
import pytest

from paper_1803_04120_gb300 import sj


def item_blocks(cell_sizes):
    """Block index within its cell of every work item (32 points a block)."""
    out = []
    for c in cell_sizes:
        out.extend(range((int(c) + 31) // 32))
    return np.asarray(out, dtype=np.uint32)


def check_tiling(blocks, world):
    n = len(blocks)
    prev = 0
    for r in range(world):
        lo, hi = sj.sj_shard_bounds(blocks, r, world)
        assert lo == prev and lo <= hi <= n
        assert lo == n or blocks[lo] == 0          # starts at a cell start
        assert hi == n or blocks[hi] == 0
        prev = hi
    assert prev == n


@pytest.mark.parametrize("seed", range(6))
def test_shard_bounds_tile_items_at_cell_starts(seed):
    rng = np.random.default_rng(seed)
    sizes = rng.integers(1, 200, size=int(rng.integers(1, 400)))
    if seed % 2:
        sizes[rng.integers(len(sizes))] = 5000    # one heavy cell spanning many items
    blocks = item_blocks(sizes)
    for world in (1, 2, 3, 5, 8, 64):
        check_tiling(blocks, world)


def test_shard_bounds_edge_cases():
    assert sj.sj_shard_bounds(np.zeros(0, np.uint32), 0, 1) == (0, 0)
    blocks = item_blocks([1000])                 # one cell: all items to one rank
    got = [sj.sj_shard_bounds(blocks, r, 4) for r in range(4)]
    assert sum(hi - lo for lo, hi in got) == len(blocks)
    assert sum(1 for lo, hi in got if hi > lo) == 1
    for bad in ((0, 0), (2, 2), (-1, 2)):
        with pytest.raises(sj.SJError):
            sj.sj_shard_bounds(blocks, bad[0], bad[1])


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, q):
    import sys
    import torch
    import torch.distributed as dist
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    from paper_1803_04120_gb300 import sj as sj_
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rng = np.random.default_rng(7)
    blocks = item_blocks(rng.integers(1, 300, size=500))
    lo, hi = sj_.sj_shard_bounds(blocks, rank, world)
    # every rank's share, gathered: the shards tile the items
    t = torch.tensor([lo, hi], dtype=torch.int64)
    allr = [torch.zeros(2, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(allr, t)
    n_own = torch.tensor([hi - lo], dtype=torch.int64)
    dist.all_reduce(n_own)
    # replica aggregation: slowest rank's time, all ranks' pairs
    ms, value = bench.replica_value(10.0 + rank, 1000, "cpu")
    q.put((rank, [tuple(x.tolist()) for x in allr], int(n_own.item()), len(blocks), ms, value))
    dist.destroy_process_group()


def test_two_ranks_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ranges, n_own, n, ms, value in res:
        assert ranges[0][0] == 0 and ranges[0][1] == ranges[1][0] and ranges[1][1] == n
        assert n_own == n
        assert ms == 11.0 and abs(value - 2 * 1000 / 0.011) < 1e-6
