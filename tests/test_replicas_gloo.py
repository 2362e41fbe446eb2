"""The multi-GPU path of bench.py is replicas only: every rank runs its own
builds, the job time is the slowest rank's and the value counts every rank's
builds. These tests run that reduction with two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 100.0 + 50.0 * rank          # rank 1 is the slow replica
    ms = bench.max_over_ranks(local_ms, dist, "cpu")
    out[rank] = (ms, bench.job_throughput(ms, steps=2, world=world), bench.job_throughput(ms, 2, world, 64))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    with mp.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [mp.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(2):
        ms, v, v64 = res[r]
        assert ms == 150.0                       # both ranks see the slowest replica
        assert abs(v - 2 * 2 / 0.150) < 1e-9     # 2 ranks x 2 builds over 150 ms
        assert abs(v64 - 64 * 2 * 2 / 0.150) < 1e-6


def test_reference_arm_other_ranks_exit_without_work():
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        workload, warmup, steps = "cluster96", 3, 2

    assert bench.run_reference(Args(), rank=1, world=2) == 0
