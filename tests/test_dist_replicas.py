"""The replica path of bench.py (N > 1) on CPU: two gloo ranks agree on the
slowest rank's time and the whole-job throughput."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_0912_3678_gb300 import dist as bd
    assert bd.env() == (world, rank, rank)
    bd.barrier()
    step_s = 0.010 * (rank + 1)                  # rank 1 is the slow one
    slow = bd.max_over_ranks(step_s)
    thr = bd.job_throughput(1000.0, step_s)
    q.put((rank, slow, thr))
    bd.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_rank():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slow, thr in res:
        assert slow == pytest.approx(0.020)
        assert thr == pytest.approx(2 * 1000.0 / 0.020)


def test_single_process_defaults():
    from paper_0912_3678_gb300 import dist as bd
    assert bd.max_over_ranks(3.5) == 3.5
    assert bd.job_throughput(10.0, 2.0) == 5.0
