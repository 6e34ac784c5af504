"""The multi-process path of the benchmark (one replica per rank, weak
scaling) on the CPU: two gloo ranks agree on the slowest rank's time and on
the whole-job rate; the reference arm runs on rank 0 only."""

import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, queue):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    r, w, local = bench.env_rank()
    dist.init_process_group("gloo", rank=r, world_size=w)
    ms = 10.0 + 5.0 * r                      # rank 1 is the slower replica
    m = bench.max_over_ranks(ms, dist, device="cpu")
    queue.put((r, w, local, m, bench.job_rate(1000, w, m)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time_and_the_job_rate():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    queue = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, queue)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(queue.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[:3] for r in res] == [(0, 2, 0), (1, 2, 1)]
    for _, _, _, m, val in res:
        assert m == 15.0 and val == pytest.approx(2 * 1000 / 0.015)


def test_single_process_and_reference_arm_on_other_ranks():
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.job_rate(500, 1, 250.0) == pytest.approx(2000.0)
    args = argparse.Namespace(n=256, nt=32, warmup=1, steps=1, gpus=2)
    assert bench.run_reference(args, 1, 2) == 0          # no work off rank 0
