"""The N > 1 path of bench.py (replicas, no collective on the data path) on two
gloo ranks on the CPU: rank setup, barrier, the max-over-ranks timing and the
whole-job rate."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    import bench
    w, r, local = bench.dist_init("gloo")
    assert (w, r, local) == (world, rank, rank)
    bench.barrier(w)
    t = bench.max_over_ranks(1.0 + rank, w)          # rank 1 is the slowest
    rate = bench.whole_job_rate(w, 1e9, t)
    out.put((rank, t, rate))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_rate():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t, rate in res:
        assert t == 2.0                      # max over ranks
        assert rate == pytest.approx(1.0)    # 2 ranks x 1e9 points / 2 s
