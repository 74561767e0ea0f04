"""The multi-GPU form is replicas only: every rank decodes its own frames and
the bench reports whole-job frames/s over the slowest rank's time.  These CPU
tests run the rank-level logic of bench.py in two gloo processes."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, times, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, local = bench._dist()
        slowest = bench.max_over_ranks(times[rank], torch.device("cpu"))
        rate = bench.job_rate(60, ws, slowest)
        q.put((r, ws, local, slowest, rate))
    finally:
        dist.destroy_process_group()


def test_job_rate_single_rank():
    assert bench.job_rate(60, 1, 1000.0) == pytest.approx(60.0)
    assert bench.job_rate(10, 1, 250.0) == pytest.approx(40.0)


@pytest.mark.parametrize("times", [(200.0, 250.0), (300.0, 120.0)])
def test_two_rank_gloo_slowest_rank_and_whole_job_rate(times):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    slow = max(times)
    for r, (rank, ws, local, slowest, rate) in enumerate(res):
        assert (rank, ws, local) == (r, 2, r)
        assert slowest == pytest.approx(slow)
        # 60 frames on each of 2 ranks over the slowest rank's time
        assert rate == pytest.approx(120 / (slow / 1e3))
