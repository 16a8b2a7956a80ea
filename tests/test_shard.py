"""Cost-balanced sharding of one batch across ranks (host logic, no GPU)."""
import json
import os

import numpy as np
import pytest

from paper_2407_09333_b300 import shard, workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_costs_are_padded_blocks_times_ops_per_block():
    lens = np.array([0, 55, 56, 64, 119, 120, 16384])
    nb = np.array([1, 1, 2, 2, 2, 3, 257])
    assert (shard.padded_blocks(lens) == nb).all()
    assert (shard.message_costs(lens, alg=2) == nb * 1412).all()
    algs = np.array([0, 1, 2, 9, 0, 1, 2], dtype=np.uint8)
    want = nb * np.array([324, 613, 1412, 0, 324, 613, 1412])
    assert (shard.message_costs(lens, algs=algs) == want).all()


@pytest.mark.parametrize("parts", [1, 2, 3, 8, 100])
def test_partition_is_contiguous_disjoint_and_balanced(parts):
    rng = np.random.default_rng(parts)
    costs = rng.integers(1, 10_000, size=5000) * rng.integers(1, 5, size=5000)
    ranges = shard.partition(costs, parts)
    assert len(ranges) == parts and ranges[0][0] == 0 and ranges[-1][1] == costs.size
    for (a, b), (c, d) in zip(ranges, ranges[1:]):
        assert b == c and a <= b
    sums = [int(costs[a:b].sum()) for a, b in ranges]
    assert sum(sums) == int(costs.sum())
    assert max(sums) <= costs.sum() / parts + costs.max()


def test_partition_edge_cases():
    assert shard.partition(np.array([], dtype=np.int64), 3) == [(0, 0)] * 3
    assert shard.partition(np.array([5]), 2) in ([(0, 0), (0, 1)], [(0, 1), (1, 1)])
    r = shard.partition(np.array([1, 1, 1, 1000]), 2)      # the heavy message alone
    assert r == [(0, 3), (3, 4)]
    with pytest.raises(ValueError):
        shard.partition(np.array([1]), 0)


def test_ragged_batch_splits_by_work_not_count():
    b = workloads.ragged(20000, seed=2)
    costs = shard.message_costs(b.lengths, algs=b.algs)
    ranges = shard.partition(costs, 4)
    works = [int(costs[a:c].sum()) for a, c in ranges]
    assert max(works) / min(works) < 1.05
    counts = [c - a for a, c in ranges]
    assert counts == [c - a for a, c in ranges] and sum(counts) == b.n


def _rank_main(rank, world, port, outdir):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import sys
    sys.path.insert(0, ROOT)
    import bench
    d = bench.Dist(world)
    try:
        desc, batch, mixed = bench.make_workload("c3", 0, 4096)    # the same batch on every rank
        a, c = shard.rank_range(batch.lengths, batch.algs, rank=d.rank, world=d.world)
        total = d.sum(float(c - a))
    finally:
        d.close()
    json.dump({"range": [a, c], "n": int(batch.n), "total": total},
              open(os.path.join(outdir, "rank%d.json" % rank), "w"))


def test_two_gloo_ranks_take_adjacent_ranges(tmp_path):
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    r = [json.load(open(tmp_path / ("rank%d.json" % k))) for k in range(2)]
    assert r[0]["range"][0] == 0 and r[0]["range"][1] == r[1]["range"][0]
    assert r[1]["range"][1] == r[0]["n"] and r[0]["total"] == r[0]["n"]
