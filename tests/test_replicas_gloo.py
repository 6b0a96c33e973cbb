"""The multi-GPU path is independent replicas (the sweep has no exchange
between GPUs): bench.py times every rank, takes the slowest with a MAX
all-reduce and reports the whole job.  Checked here with two gloo ranks on
the CPU (no GPU, no NCCL)."""
import importlib.util
import os
import socket

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _rank(rank, ws, port, out):
    import torch.distributed as dist

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=ws)
    try:
        b = _bench()
        ms = [3.0, 5.0][rank]  # the second replica is slower
        ms_max = b._max_over_ranks(ms, ws, "cpu")
        out[rank] = (ms_max, b._job_value(ws, 1000, 10, ms_max))
    finally:
        dist.destroy_process_group()


def test_two_replicas_report_the_slowest_and_the_whole_job():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = torch.multiprocessing.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    # both ranks see the slower replica's 5 ms; 2 x 1000 cells x 10 steps in 5 ms = 4 MLUPS
    assert out[0] == out[1] == (5.0, 4.0)


def test_one_replica_needs_no_collective():
    b = _bench()
    assert b._max_over_ranks(2.5, 1, "cpu") == 2.5
    assert b._job_value(1, 1000, 10, 2.5) == 4.0
