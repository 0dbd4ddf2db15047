"""Multi-GPU runs are independent replicas (the step has no exchange on one
mesh per GPU): the benchmark's host logic -- barrier, the maximum of the
ranks' times, the whole-job aggregate -- checked with two gloo ranks on CPU."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, times, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    bench.barrier(world)
    ms = bench.max_over_ranks(times[rank], world)
    faces = world * 10 * 1000            # whole job: every rank advanced 10 steps of 1000 faces
    out[rank] = (ms, faces / (ms * 1e-3) / 1e6)
    dist.destroy_process_group()


def test_two_gloo_replicas_report_the_slowest_rank():
    import torch.multiprocessing as mp
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    times = [12.5, 17.0]
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank, args=(r, 2, port, times, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == out[1]
    ms, value = out[0]
    assert ms == 17.0
    assert value == pytest.approx(2 * 10 * 1000 / 17.0e-3 / 1e6)
