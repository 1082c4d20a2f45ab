"""The benchmark's multi-rank path on CPU (gloo, two ranks): each rank times its
own independent frame stream; the job's throughput is all ranks' vertices
over the slowest rank's time (weak scaling), and only rank 0 reports."""
import os

import torch.multiprocessing as mp


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [12.5, 20.0][rank]
    vertices = [1_000_000, 1_500_000][rank]
    q.put((rank,) + bench.reduce_ranks(ms, float(vertices)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_report_slowest_time_and_total_vertices():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 2000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, v in got:
        assert ms == 20.0 and v == 2_500_000.0


def test_single_rank_is_unchanged():
    import bench
    assert bench.reduce_ranks(3.0, 7.0) == (3.0, 7.0)
