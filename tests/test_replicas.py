"""bench.py with N > 1 runs N independent replicas (the method is not sharded across GPUs in this build):
every rank times its own steps and the job's time is the slowest rank's.  The aggregation runs here as
two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, port, totals, out):
    import torch
    import torch.distributed as tdist
    sys.path.insert(0, ROOT)
    import bench
    tdist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=2)
    try:
        tdist.barrier()
        job_ms, value = bench.replica_throughput(totals[rank], 1000, 5, 2, torch.device("cpu"))
        out[rank] = (job_ms, value)
    finally:
        tdist.destroy_process_group()


def test_replica_throughput_takes_the_slowest_rank():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    totals = [10.0, 12.5]
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, port, totals, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    for r in range(2):
        job_ms, value = out[r]
        assert job_ms == 12.5
        assert value == pytest.approx(2 * 1000 * 5 / 0.0125)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    job_ms, value = bench.replica_throughput(4.0, 100, 2, 1, None)
    assert job_ms == 4.0 and value == pytest.approx(100 * 2 / 0.004)
