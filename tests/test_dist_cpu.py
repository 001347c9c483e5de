"""Multi-process (weak-scaling replica) aggregation of bench.py on CPU.

Each rank evaluates its own population; the job's time is the slowest
rank's and the throughput counts every rank's candidates.  Two gloo ranks
on 127.0.0.1 check that reduction without a GPU.
"""
import os

import torch.multiprocessing as mp


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = 1.5 + rank  # rank 1 is slower
    tmax = bench.max_over_ranks(t, world, device="cpu")
    q.put((rank, tmax, bench.job_throughput(256, 3, tmax, world)))
    dist.destroy_process_group()


def test_two_rank_max_and_throughput():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [2.5, 2.5]
    assert abs(res[0][2] - 2 * 256 * 3 / 2.5) < 1e-9


def test_single_rank_passthrough():
    import bench
    assert bench.max_over_ranks(3.0, 1) == 3.0
    assert bench.job_throughput(256, 2, 4.0, 1) == 128.0
