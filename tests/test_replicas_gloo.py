"""Multi-GPU is replicas only (streams are independent, no data-path collective).
This checks the host logic bench.py runs under torchrun, with world_size-2 gloo
ranks on the CPU: the max-over-ranks timing, the whole-job throughput and the
per-rank seeds."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 10.0 + 5.0 * rank          # rank 1 is the slow one
        ms = bench.max_over_ranks(local_ms)
        q.put((rank, ms, bench.rank_seed(1200, rank)))
    finally:
        dist.destroy_process_group()


def test_two_replicas_max_time_and_seeds():
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
    assert [r[1] for r in res] == [15.0, 15.0]          # every rank sees the slowest time
    assert res[0][2] != res[1][2]                         # replicas draw different streams


def test_whole_job_throughput_counts_all_ranks():
    sys.path.insert(0, ROOT)
    import bench
    # 2 ranks x 1000 samples per step x 10 steps = 20000 samples in 1 ms -> 20 Msamples/s
    assert bench.whole_job_msps(1000, 2, 10, 1.0) == pytest.approx(20.0)
    assert bench.max_over_ranks(3.5) == 3.5               # single process: no collective
