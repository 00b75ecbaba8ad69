"""The multi-GPU bench path on CPU: two gloo ranks, each solving its own copy
(weak scaling, no collective on the data path); the job's time is the slowest
rank and its work the sum over ranks."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r "took" 100 (r + 1) ms for 1000 (r + 1) iterations
    t, n = bench.reduce_max_sum([100.0 * (rank + 1), 1000.0 * (rank + 1)], "cpu")
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, t, n))


def test_two_rank_aggregation_gloo():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=5) for _ in range(2))
    for rank, t, n in res:
        assert t == 200.0 and n == 3000.0


def test_single_process_aggregation_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max_sum([12.5, 7.0], "cpu") == (12.5, 7.0)
