"""The multi-GPU path of bench.py is replicas: every rank solves its own copy of the cell, with
no collective in the data path.  Its host logic runs here on CPU with gloo, world size 2: the
whole-job value is the slowest rank's time over world x steps ground states, and only rank 0
runs and prints the reference arm."""
import contextlib
import io
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        step_ms = [100.0 + 50.0 * rank, 200.0]   # rank 1 is the slower replica
        total, value = bench.whole_job_value(step_ms, 2, world, "cpu")
        dist.barrier()
        q.put((rank, total, value))
    finally:
        dist.destroy_process_group()


def test_whole_job_value_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, total, value in out:
        assert total == 350.0                        # max over ranks of 300 and 350 ms
        assert value == pytest.approx(0.35 / (2 * 2))  # 2 ranks x 2 steps ground states


def test_whole_job_value_single_rank():
    total, value = bench.whole_job_value([400.0, 600.0], 2, 1, "cpu")
    assert total == 1000.0 and value == pytest.approx(0.5)


def test_reference_arm_other_ranks_exit_quietly():
    class Args:
        steps, warmup, gpus = 1, 0, 2
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        assert bench.reference_arm(Args(), rank=1, world=2) == 0
    assert buf.getvalue() == ""
