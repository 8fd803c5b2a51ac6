"""The multi-rank path of bench.py on CPU: two gloo ranks (replicas) agree on
the slowest rank's time and on the whole-job DOF/s; the reference arm prints
only on rank 0."""
import contextlib
import io
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    seconds = 1.0 + rank  # rank 1 is slower
    t = bench.reduce_max(seconds, "cpu")
    v = bench.weak_scaling_value(world, 1000, 10, t)
    dist.barrier()
    out[rank] = (t, v)
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    assert res[0] == res[1] == (2.0, 2 * 1000 * 10 / 2.0)


def test_reference_arm_prints_only_on_rank_zero(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(bench.parse_args.__wrapped__() if hasattr(bench.parse_args, "__wrapped__") else
                            type("A", (), dict(steps=1, warmup=0, gpus=2))())
    assert buf.getvalue() == ""


def test_single_process_reduce_is_identity():
    import bench
    assert bench.reduce_max(3.5) == 3.5
    assert bench.weak_scaling_value(1, 10, 2, 4.0) == 5.0
