"""The N-GPU benchmark path (replicas, one process per GPU) on CPU: two gloo
ranks agree on the job's time (the slowest rank's) and value (all ranks'
updates over it), and each rank updates its own graph."""
import multiprocessing as mp
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.job_ms(100.0 + 50.0 * rank, dist, device="cpu")     # rank 1 is the slower one
    value = bench.job_value(1000, world, ms)
    dist.barrier()
    q.put((rank, ms, value, bench.rank_seed(rank)))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, ms0, v0, s0), (r1, ms1, v1, s1) = out
    assert ms0 == ms1 == 150.0
    assert v0 == v1 == 2 * 1000 / 0.150
    assert s0 != s1


def test_single_rank_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_ms(42.0, None) == 42.0
    assert bench.job_value(100, 1, 50.0) == 2000.0
