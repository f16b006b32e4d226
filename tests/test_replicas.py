"""Whole-job timing of independent replicas, on two CPU processes over gloo: every rank sees
the slowest rank's time, and the job rate counts every rank's units over it."""
import os
import socket

import pytest
import torch
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    from paper_2604_01844_gb300 import replicas as R

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert R.world() == world
        ms = 10.0 + 5.0 * rank  # rank 1 is slower
        slow = R.slowest(ms)
        out[rank] = (slow, R.job_rate(1000.0, slow, world))
    finally:
        dist.destroy_process_group()


def test_two_replicas_gloo():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
        for r in range(2):
            slow, rate = out[r]
            assert slow == 15.0
            assert rate == pytest.approx(2 * 1000.0 / 15e-3)


def test_single_process_is_identity():
    from paper_2604_01844_gb300 import replicas as R

    assert R.world() == 1
    assert R.slowest(3.5) == 3.5
    assert R.job_rate(10.0, 2.0, 1) == pytest.approx(5000.0)
