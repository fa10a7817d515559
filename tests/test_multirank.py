"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): the slowest rank's time
and every rank's work define the whole-job throughput ("replicas only": no data-path
collective exists)."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        local_seconds = [0.5, 2.0][rank]
        m = bench.reduce_max(local_seconds)
        v = bench.whole_job_value(1e9, 10, m, world)
        out[rank] = (m, v)
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation_takes_the_slowest_rank():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(2):
        m, v = out[r]
        assert m == 2.0
        assert v == pytest.approx(2 * 1e9 * 10 / 2.0 / 1e9)


def test_single_process_aggregation_is_identity():
    import bench
    assert bench.reduce_max(1.25) == 1.25
    assert bench.whole_job_value(2e9, 5, 2.0, 1) == pytest.approx(5.0)
