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
