"""Host logic of the multi-rank paths, on the CPU: the shard rules of
sj_selfjoin_shard_device (ranges of work items cut at cell starts, balanced
by query blocks or by estimated cost) and the replica aggregation of
bench.py, with world_size 2 gloo process groups."""
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


def cell_costs(rng, sizes):
    """Per-item costs of the shape the device estimates, K (q + 20) + 2000,
    with the candidate count K of a cell growing with its population (a
    dense cell has dense neighbours): skewed, as on clustered data."""
    blocks, cost = [], []
    for c in sizes:
        K = int(c) * int(rng.integers(3, 30))
        for b in range((int(c) + 31) // 32):
            q = min(32, int(c) - 32 * b)
            blocks.append(b)
            cost.append(K * (q + 20) + 2000)
    return np.asarray(blocks, dtype=np.uint32), np.asarray(cost, dtype=np.uint64)


def shard_costs(blocks, cost, world, rule):
    out, prev = [], 0
    for r in range(world):
        lo, hi = rule(r)
        assert lo == prev and lo <= hi <= len(blocks)
        assert lo == len(blocks) or blocks[lo] == 0
        prev = hi
        out.append(int(cost[lo:hi].sum()))
    assert prev == len(blocks)
    return out


@pytest.mark.parametrize("seed", range(6))
def test_cost_bounds_tile_and_balance_skewed_cells(seed):
    rng = np.random.default_rng(100 + seed)
    sizes = np.concatenate([rng.integers(1, 20, size=3000), rng.integers(200, 3000, size=12)])
    rng.shuffle(sizes)
    blocks, cost = cell_costs(rng, sizes)
    starts = np.flatnonzero(blocks == 0)
    cell_cost = np.add.reduceat(cost, starts)
    total = int(cost.sum())
    for world in (2, 3, 4, 8):
        by_cost = shard_costs(blocks, cost, world,
                              lambda r: sj.sj_shard_bounds_cost(blocks, cost, r, world))
        by_blocks = shard_costs(blocks, cost, world, lambda r: sj.sj_shard_bounds(blocks, r, world))
        assert sum(by_cost) == total == sum(by_blocks)
        # each bound is off its target by at most half a cell
        assert max(by_cost) <= total / world + int(cell_cost.max())


def test_cost_bounds_beat_block_bounds_on_front_loaded_work():
    # the first half of the items (by count) carries almost all the cost:
    # equal item counts put it on one rank, equal costs spread it
    rng = np.random.default_rng(3)
    heavy = [64] * 200                 # 2 items each, expensive
    light = [32] * 400                 # 1 item each, cheap
    blocks = item_blocks(heavy + light)
    cost = np.concatenate([np.full(400, 10**6), np.full(400, 10)]).astype(np.uint64)
    by_blocks = shard_costs(blocks, cost, 2, lambda r: sj.sj_shard_bounds(blocks, r, 2))
    by_cost = shard_costs(blocks, cost, 2, lambda r: sj.sj_shard_bounds_cost(blocks, cost, r, 2))
    assert max(by_blocks) >= 0.99 * int(cost.sum())
    assert max(by_cost) <= 0.51 * int(cost.sum())


def test_cost_bounds_edge_cases():
    blocks = item_blocks([10, 10, 10, 10])
    cost = np.array([5, 1, 1, 1], dtype=np.uint64)
    assert [sj.sj_shard_bounds_cost(blocks, cost, r, 2) for r in range(2)] == [(0, 1), (1, 4)]
    # a heavy cell of three items straddling the target: the nearer start
    hb = item_blocks([10, 96, 10])
    hc = np.array([1, 5, 5, 5, 20], dtype=np.uint64)
    assert [sj.sj_shard_bounds_cost(hb, hc, r, 2) for r in range(2)] == [(0, 4), (4, 5)]
    hc = np.array([20, 5, 5, 5, 1], dtype=np.uint64)
    assert [sj.sj_shard_bounds_cost(hb, hc, r, 2) for r in range(2)] == [(0, 1), (1, 5)]
    zero = np.zeros(4, dtype=np.uint64)
    got = [sj.sj_shard_bounds_cost(blocks, zero, r, 3) for r in range(3)]
    assert got[0][0] == 0 and got[-1][1] == 4
    assert sj.sj_shard_bounds_cost(np.zeros(0, np.uint32), np.zeros(0, np.uint64), 0, 1) == (0, 0)
    with pytest.raises(sj.SJError):
        sj.sj_shard_bounds_cost(blocks, cost, 2, 2)


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
    sizes = np.concatenate([rng.integers(1, 300, size=500), [4000, 6000]])
    rng.shuffle(sizes)
    blocks, cost = cell_costs(rng, sizes)
    lo, hi = sj_.sj_shard_bounds_cost(blocks, cost, rank, world)
    # every rank's share, gathered: the shards tile the items and their
    # estimated costs are balanced
    t = torch.tensor([lo, hi, int(cost[lo:hi].sum())], dtype=torch.int64)
    allr = [torch.zeros(3, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(allr, t)
    n_own = torch.tensor([hi - lo], dtype=torch.int64)
    dist.all_reduce(n_own)
    # replica aggregation: slowest rank's time, all ranks' pairs
    ms, value = bench.replica_value(10.0 + rank, 1000, "cpu")
    cell_max = int(np.add.reduceat(cost, np.flatnonzero(blocks == 0)).max())
    q.put((rank, [tuple(x.tolist()) for x in allr], int(n_own.item()), len(blocks), ms, value,
           int(cost.sum()), cell_max))
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
    for rank, ranges, n_own, n, ms, value, total, cell_max in res:
        assert ranges[0][0] == 0 and ranges[0][1] == ranges[1][0] and ranges[1][1] == n
        assert n_own == n
        assert ranges[0][2] + ranges[1][2] == total
        assert max(ranges[0][2], ranges[1][2]) <= total / 2 + cell_max
        assert ms == 11.0 and abs(value - 2 * 1000 / 0.011) < 1e-6
