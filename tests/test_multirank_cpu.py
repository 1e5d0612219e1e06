"""The N > 1 host logic of the benchmark (replicas, max over ranks) with two gloo ranks on CPU."""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    seed = bench.replica_seed(7, rank)
    # each replica's "time" differs; the reported value is the maximum over ranks
    vals = bench.max_over_ranks([1.0 + rank, 10.0 - rank])
    from paper_2509_11890_gb300 import inputs
    inst = inputs.maxcut_kron(4, seed)
    out.put((rank, seed, vals, int(inst["adjacency"].sum())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_replicas_and_max():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29517
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, v0, e0), (r1, s1, v1, e1) = res
    assert (s0, s1) == (7, 8)                  # distinct instances per replica
    assert v0 == v1 == [2.0, 10.0]             # element-wise max over the two ranks
    assert e0 > 0 and e1 > 0


def test_partition_batch_is_balanced_and_complete():
    sys.path.insert(0, ROOT)
    import bench
    from paper_2509_11890_gb300 import inputs
    orders = [i["d"] for i in inputs.batch_maxcut(64, 0)]
    for world in (1, 2, 3, 8):
        shards = bench.partition_batch(orders, world, 64)
        flat = sorted(j for sh in shards for j in sh)
        assert flat == list(range(64))                      # every instance exactly once
        loads = [sum(orders[j] for j in sh) for sh in shards]
        # LPT on costs proportional to d: the spread is at most one instance
        assert max(loads) - min(loads) <= max(orders)
    assert bench.partition_batch([6, 7, 11], 2, 64) == [[2], [0, 1]]


def _gather_worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    orders = [6, 9, 11, 7, 8, 10, 6]
    mine = bench.partition_batch(orders, world, 64)[rank]
    res = bench.gather_results({j: (0, float(orders[j]), 4) for j in mine}, world)
    out.put((rank, mine, sorted(res.items())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_gather_a_batch():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_gather_worker, args=(r, 2, 29531, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, m0, g0), (_, m1, g1) = res
    assert sorted(m0 + m1) == list(range(7)) and not set(m0) & set(m1)
    assert g0 == g1 and [k for k, _ in g0] == list(range(7))   # both ranks see every result
