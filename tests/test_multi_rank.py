"""The benchmark's multi-rank path, on the CPU with two gloo ranks.

Messages are independent, so ranks hash disjoint shards and talk only to
agree on the timed region: a barrier on both sides, the slowest rank's time
and the sum of every rank's bytes.  These tests run that plumbing with the
gloo backend (no GPU): the reductions, the whole-job rate, the per-rank
shards, and the reference arm under torchrun, where rank 0 alone works and
prints and the other rank exits 0.
"""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, outdir):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench

    d = bench.Dist(world)
    try:
        d.barrier()
        res = {
            "rank": d.rank, "world": d.world, "backend": d.pg.get_backend(),
            "max": d.max(float(rank + 1)),
            "sum": d.sum(float(rank + 1)),
            # rank r hashed 100 (r + 1) units in (r + 1) seconds
            "rate": bench.job_rate(d, 100.0 * (rank + 1), float(rank + 1)),
        }
        desc, batch, mixed = bench.make_workload("c3", d.rank, 256)
        res["shard_bytes"] = int(batch.total_bytes)
        res["shard_head"] = batch.packed[:64].tolist()
        d.barrier()
    finally:
        d.close()
    with open(os.path.join(outdir, "rank%d.json" % rank), "w") as f:
        json.dump(res, f)


def test_two_gloo_ranks_reduce_and_shard(tmp_path):
    import torch.multiprocessing as mp

    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / ("rank%d.json" % r))) for r in range(world)]
    for r, x in enumerate(res):
        assert x["rank"] == r and x["world"] == world and x["backend"] == "gloo"
        assert x["max"] == 2.0          # slowest rank's time
        assert x["sum"] == 3.0          # every rank's units
        assert x["rate"] == pytest.approx(300.0 / 2.0)
    # disjoint synthetic shards: different bytes on each rank
    assert res[0]["shard_head"] != res[1]["shard_head"]
    assert res[0]["shard_bytes"] != res[1]["shard_bytes"]


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        assert k not in os.environ or os.environ[k] in ("0", "1")
    d = bench.Dist(1)
    assert d.pg is None and d.world == 1
    assert d.max(3.5) == 3.5 and d.sum(3.5) == 3.5
    assert bench.job_rate(d, 10.0, 4.0) == 2.5
    assert bench.shard_seed(2, 0) != bench.shard_seed(2, 1)


def test_reference_arm_under_torchrun_prints_once(tmp_path, oracle_mod):
    env = dict(os.environ)
    env.pop("CUDA_VISIBLE_DEVICES", None)
    env["CUDA_VISIBLE_DEVICES"] = ""          # CPU only: gloo ranks
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "c1",
           "--gpus", "2", "--steps", "2", "--warmup", "3"]
    p = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-3000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, p.stdout
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["value"] > 0 and line["unit"] == "GB/s"
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0
    assert np.isfinite(line["ms_per_step"])
