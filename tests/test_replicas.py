"""The multi-GPU bench path is replicas only (independent solves per rank, no
data-path collective): the timed region's max over ranks and the whole-job
value, exercised with 2 gloo ranks on CPU."""
import os
import socket

import pytest


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
    ms = bench.max_over_ranks(1000.0 + 250.0 * rank, world, device="cpu")
    q.put((rank, ms, bench.replica_value(world, 3, ms)))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_value_with_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # both ranks see the slowest rank's time; value counts both ranks' solves
    assert [o[1] for o in out] == [1250.0, 1250.0]
    assert out[0][2] == pytest.approx(2 * 3 / 1.25)


def test_single_rank_needs_no_collective():
    import bench
    assert bench.max_over_ranks(42.0, 1) == 42.0
    assert bench.replica_value(1, 2, 500.0) == pytest.approx(4.0)
