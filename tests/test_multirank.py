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


def _split_rank_main(rank, world, port, out_dir):
    """The two-GPU expectation split (Sec. IV-B's two sweep directions on two
    ranks) with the oracle standing in for the device work: rank r runs only
    the sweeps of its direction (top-down: 0 and 2, bottom-up: 1 and 3),
    the regions are exchanged by libpeps.exchange_env_regions (one broadcast
    per part), then every rank evaluates the strips from both parts."""
    sys.path.insert(0, ROOT)
    import pickle

    import torch
    import torch.distributed as dist

    import synth
    from oracle import bmps, expectation
    from paper_2006_15234_gb300 import libpeps
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ket = synth.random_peps(4, 3, 2, 2, "f64", "normal", 83)
        terms = synth.tfi_terms(4, 3, 1.0, 3.0)
        real_sweep = bmps.sweep
        # the sweeps of Sec. IV-B: directions 0 / 1 top-down / bottom-up on the
        # lattice, 2 / 3 on its transpose (vertical terms); this rank's part only
        lattices = {0: ket, 2: bmps.transpose_lattice(ket)}
        mine, ran = {}, []
        for direction in (rank, rank + 2):
            lat = lattices[direction - direction % 2]
            if direction % 2:
                lat = bmps.flip_vertical(lat)
            ran.append(direction)
            mine[direction] = real_sweep(lat, lat, 4, 4, 1, 5, direction, len(lat) - 2)
        blob = pickle.dumps(mine)
        sizes = [None] * world
        dist.all_gather_object(sizes, len(blob))
        views = [torch.zeros(n, dtype=torch.uint8) for n in sizes]
        views[rank][:] = torch.frombuffer(bytearray(blob), dtype=torch.uint8)
        libpeps.exchange_env_regions(views)
        both = {}
        for v in views:
            both.update(pickle.loads(v.numpy().tobytes()))
        bmps.sweep = lambda ket_, bra_, m, p, q, seed, direction, last, *a: both[direction]
        e = expectation.energy(ket, terms, 4, 4, 1, 5)
        bmps.sweep = real_sweep
        ref = expectation.energy(ket, terms, 4, 4, 1, 5)
        gathered = [None] * world
        dist.all_gather_object(gathered, {"e": e, "ref": ref, "ran": sorted(ran)})
        if rank == 0:
            import json
            with open(os.path.join(out_dir, "split.json"), "w") as f:
                json.dump(gathered, f)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_split_the_expectation_sweeps(tmp_path):
    """Each rank computes only its sweep direction; after the exchange both
    ranks hold the single-rank energy exactly."""
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_split_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    import json
    res = json.load(open(tmp_path / "split.json"))
    assert res[0]["ran"] == [0, 2] and res[1]["ran"] == [1, 3]
    for r in res:
        assert r["e"] == r["ref"]
    assert res[0]["e"] == res[1]["e"]
    del torch
