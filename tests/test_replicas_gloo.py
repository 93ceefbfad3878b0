"""The multi-rank (replica) host logic of bench.py on CPU: two gloo ranks reduce their step
times to the slowest rank's, and the reference leg runs on rank 0 only."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    out[rank] = bench.max_over_ranks(1.5 + rank)
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    import torch.multiprocessing as mp
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, start_method="spawn", join=True)
    assert dict(out) == {0: 2.5, 1: 2.5}


def test_max_over_ranks_single_process():
    import bench
    assert bench.max_over_ranks(3.25) == 3.25


def test_reference_leg_only_on_rank0():
    import bench

    class A:
        N, warmup, steps, gpus = 16, 0, 0, 2

    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(A(), rank=1)
    assert buf.getvalue() == ""
