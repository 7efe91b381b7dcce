"""bench.py's N > 1 path on CPU: 2 gloo ranks, the job time is the slowest
rank's, and the value counts the units of every rank (equal for replicas,
unequal for the shards of a batch, whose members each rank draws alone)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 100.0 if rank == 0 else 250.0          # rank 1 is the slow one
    value, ms = bench.aggregate(local_ms, 1_000_000, world)
    # a batch shard: the ranks scored different edge counts
    v2, ms2 = bench.aggregate(local_ms, 3_000 if rank == 0 else 5_000, world)
    q.put((rank, value, ms, v2, ms2))
    dist.destroy_process_group()


def test_replica_aggregation_two_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, value, ms, v2, ms2 in res:
        assert ms == 250.0 and ms2 == 250.0            # max over ranks
        assert value == pytest.approx(2 * 1_000_000 / 0.25)
        assert v2 == pytest.approx(8_000 / 0.25)       # sum of the ranks' units


def test_batch_shards_are_the_members_of_a_larger_batch():
    """Rank r's batch members [rG, (r+1)G) are drawn alone and equal that slice of one
    2G-graph batch: the shards are disjoint and rank 0's is the 1-GPU batch."""
    import graphgen
    G = 64
    whole = graphgen._batch_sizes(2 * G, 500, 200_000, 4)
    assert graphgen._batch_sizes(G, 500, 200_000, 4) == whole[:G]
    assert graphgen._batch_sizes(G, 500, 200_000, 4, first=G) == whole[G:]


def test_single_rank_aggregation():
    import bench
    value, ms = bench.aggregate(50.0, 1000, 1)
    assert ms == 50.0 and value == pytest.approx(20000.0)
