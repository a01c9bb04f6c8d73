"""The multi-GPU form of the path is replicas only (one independent projection per GPU, no
collective on the data path): the benchmark's job time is the maximum over ranks and its
throughput the sum of the replicas' work over that time.  These checks run the host logic as
two gloo ranks on the CPU."""

import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    import argparse

    import bench
    # rank r contributes (r + 1.5, 10 - r): the job time is the element-wise maximum on every rank
    got = bench.max_over_ranks([rank + 1.5, 10.0 - rank])
    # the reference arm runs on rank 0 only; other ranks return at once without work
    ref = bench.run_reference(argparse.Namespace(steps=1, warmup=3), rank, world) if rank else None
    torch.distributed.barrier()
    torch.distributed.destroy_process_group()
    out.put((rank, got, ref))


def test_two_gloo_ranks_take_the_maximum_time_and_only_rank0_reports():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(world):
        r, got, ref = q.get(timeout=120)
        res[r] = (got, ref)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(world):
        assert res[r][0] == [world - 1 + 1.5, 10.0]
    assert res[1][1] == 0


def test_job_throughput_counts_every_replica():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_mpts(1, 1_000_000, 1.0) == pytest.approx(1000.0)
    assert bench.job_mpts(4, 1_000_000, 2.0) == pytest.approx(2000.0)
    assert bench.max_over_ranks([3.0, 1.0]) == [3.0, 1.0]      # no process group: identity
