"""Multi-rank aggregation of the benchmark (independent replicas), two gloo ranks on CPU.

With N GPUs the benchmark runs N independent replicas; the whole-job time is the slowest
rank's timed region and the value counts every rank's bytes.  This runs the same
aggregation functions over a real two-process gloo group.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 10.0 + 5.0 * rank            # rank 1 is the slowest
    job = bench.job_time_ms(local_ms, world, "cpu")
    val = bench.job_value_gbs(480 * 1048576, 100, world, job)
    out[rank] = (job, val)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replica_aggregation():
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0
    expect = 480 * 1048576 * 100 * 2 / 15e-3 / 1e9
    assert abs(res[0][1] - expect) < 1e-9 * expect and res[0][1] == res[1][1]
