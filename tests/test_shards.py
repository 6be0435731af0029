"""Replica sharding of the bench's serving stream and batched mix: each rank
takes a round-robin share of the independent instances (no data-path
collective); the shares partition the whole workload, and the per-rank
result lists merge back into the global order.  Exercised with two gloo
ranks on CPU, with the stored oracle results of the batched mix standing in
for the per-instance results."""
import json
import os
import socket

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    with open(os.path.join(ROOT, "tests", "golden", "batch256_oracle.json")) as f:
        gold = {r["i"]: r["delta"] for r in json.load(f)["instances"]}
    mine = bench.shard(range(256), rank, world)
    # this rank's "results": the objective of each of its instances
    results = [(i, gold[i]) for i in mine]
    parts = [None] * world
    dist.all_gather_object(parts, results)
    merged = bench.merge_shards(parts)
    total = bench.all_reduce_sum([len(mine)], world, device="cpu")[0]
    q.put((rank, mine, merged, total))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_partition_the_mix_and_merge_in_order():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    shares = [set(o[1]) for o in out]
    assert shares[0].isdisjoint(shares[1]) and shares[0] | shares[1] == set(range(256))
    with open(os.path.join(ROOT, "tests", "golden", "batch256_oracle.json")) as f:
        gold = [(r["i"], r["delta"]) for r in sorted(json.load(f)["instances"],
                                                     key=lambda r: r["i"])]
    for _, _, merged, total in out:
        assert merged == gold and total == 256


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_shard_and_merge_round_trip(world):
    import bench
    items = list(range(101))
    parts = [bench.shard(items, r, world) for r in range(world)]
    assert sum(len(p) for p in parts) == len(items)
    assert bench.merge_shards(parts) == items
    assert max(len(p) for p in parts) - min(len(p) for p in parts) <= 1


def test_fifo_latency_and_percentiles():
    import bench
    # arrivals 0, 1, 2 s; service 2 s each: waits of 0, 1, 2 s
    lat = bench.fifo_latencies_ms([0.0, 1.0, 2.0], [2.0, 2.0, 2.0])
    assert lat == [2000.0, 3000.0, 4000.0]
    assert bench.pct(lat, 50) == 3000.0 and bench.pct([], 50) is None
