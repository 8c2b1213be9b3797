"""The multi-rank host logic of the benchmark on CPU: two `gloo` ranks
(world size 2, rendezvous on 127.0.0.1), no data-path collective.  A
boundary sweep shards by replication (weak scaling: every rank contracts
its own PEPS replica); the batched einsumsvd splits ONE batch of 512
independent instances over the ranks by longest-processing-time-first on
each instance's flop count (strong scaling).  The one collective is the
maximum of the per-rank step time.  Checked here: that maximum reaches
every rank, the two ranks' instance sets are disjoint and cover the batch,
their loads differ by under 1 %, the replicas' seeds differ (and so do their
PEPS), and the whole-job value counts the work of both ranks over the
slowest rank's time."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    import synth
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        step_ms = 10.0 + 5.0 * rank                    # rank 1 is the slow one
        slowest = bench.max_over_ranks(step_ms, world, "cpu")
        cfg3 = synth.config("c3")
        costs = bench.batched_costs(cfg3, False)
        ids = bench.lpt_shard(costs, world)[rank]
        load = sum(costs[i] for i in ids)
        cfg5 = synth.config("c2")
        seed = bench.replica_seed(cfg5, rank)
        site = synth.random_peps(cfg5.nrow, cfg5.ncol, cfg5.d, cfg5.D, cfg5.dtype, cfg5.dist, seed)[1][1]
        gathered = [None] * world
        dist.all_gather_object(gathered, {"slowest": slowest, "ids": ids, "seed": seed, "load": load,
                                          "n": len(costs), "site_sum": float(np.abs(site).sum())})
        if rank == 0:
            import json
            with open(os.path.join(out_dir, "result.json"), "w") as f:
                json.dump(gathered, f)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_the_workloads(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    import json
    res = json.load(open(tmp_path / "result.json"))
    assert [r["slowest"] for r in res] == [15.0, 15.0]
    ids0, ids1 = set(res[0]["ids"]), set(res[1]["ids"])
    assert not ids0 & ids1 and ids0 | ids1 == set(range(res[0]["n"]))
    loads = [r["load"] for r in res]
    assert max(loads) / min(loads) - 1.0 < 0.01
    assert res[0]["seed"] != res[1]["seed"] and res[0]["site_sum"] != res[1]["site_sum"]
    sys.path.insert(0, ROOT)
    import bench
    flops = 2.0e12
    assert bench.whole_job_value(world, flops, 15.0) == pytest.approx(world * flops / 15e-3 / 1e12)
    assert bench.whole_job_value(1, flops, 15.0) == pytest.approx(flops / 15e-3 / 1e12)
    assert bench.max_over_ranks(3.5, 1) == 3.5
    del torch


def test_lpt_shard_properties():
    """LPT on its own: a deterministic partition covering every item once,
    its makespan within 4/3 of the lower bound max(mean load, largest item)."""
    sys.path.insert(0, ROOT)
    import bench
    rng = np.random.default_rng(3)
    for world in (1, 2, 3, 4, 8):
        costs = list(rng.pareto(1.5, 300) + 0.1)
        parts = bench.lpt_shard(costs, world)
        assert parts == bench.lpt_shard(costs, world)
        assert sorted(i for p in parts for i in p) == list(range(300))
        loads = [sum(costs[i] for i in p) for p in parts]
        lower = max(sum(costs) / world, max(costs))
        assert max(loads) <= 4.0 / 3.0 * lower + 1e-9
