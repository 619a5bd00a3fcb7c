"""The multi-GPU path of bench.py is independent replicas: value = samples of all ranks over
the slowest rank's time.  Checked with two gloo ranks on the CPU (no GPU, no data-path
collective)."""
import os
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    value, ms = bench.aggregate_replicas(10.0 + 5.0 * rank, 1e6, world)   # rank 1 is slower
    q.put((rank, value, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, ms in out:
        assert ms == 15.0                          # the slowest rank's time on every rank
        assert abs(value - 2 * 1e6 / 15e-3) < 1e-6 * value


def test_single_process_is_its_own_replica():
    sys.path.insert(0, ROOT)
    import bench
    value, ms = bench.aggregate_replicas(4.0, 1e6, 1)
    assert ms == 4.0 and abs(value - 2.5e8) < 1e-3
