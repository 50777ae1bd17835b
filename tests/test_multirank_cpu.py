"""The N > 1 path of bench.py on the CPU: two gloo ranks (127.0.0.1).

bench.py runs independent replicas on N GPUs (the workload is one device stack,
whose domain is not split): the only cross-rank operations are the barrier
around the timed region and the max-over-ranks of the elapsed time.  These
tests run exactly those helpers with world size 2 on the gloo backend.
"""
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench.dist_env()
    bench.barrier(ws)
    t = bench.reduce_max(10.0 + rank, ws)     # ranks report different elapsed times
    bench.barrier(ws)
    q.put((r, ws, t))
    dist.destroy_process_group()


def test_two_rank_max_and_barrier():
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
    assert res == [(0, 2, 11.0), (1, 2, 11.0)]


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(3.5, 1) == 3.5
    bench.barrier(1)


def _reference_worker(rank, world, port, q):
    """`--impl reference` under two ranks: rank 1 exits at once without output."""
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import bench

    class A:
        steps, warmup, cpu_seconds = 1, 3, 0.01
    if rank == 1:
        bench.run_reference(A, world, rank)
        q.put((rank, "no output"))


@pytest.mark.slow
def test_reference_arm_other_ranks_do_nothing():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    p = ctx.Process(target=_reference_worker, args=(1, 2, _free_port(), q))
    p.start()
    p.join(60)
    assert p.exitcode == 0 and q.get(timeout=10) == (1, "no output")
