"""The multi-process path of bench.py on CPU: two gloo ranks, each timing
its own replica; the job time is the maximum over ranks and the job value
counts the cells of every rank (weak scaling, no data-path collective)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        my_seconds = 1.0 + rank          # rank 1 is the slow replica
        bench.barrier(ws)
        t = bench.max_over_ranks(ws, my_seconds, device="cpu")
        out[rank] = (t, bench.job_value(ws, 1000, 10, t))
        bench.barrier(ws)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_replica():
    ws = 2
    port = _free_port()
    # spawn, not fork: the test process may already hold threads (or a CUDA context)
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    assert res[0] == res[1]
    t, value = res[0]
    assert t == 2.0
    assert value == pytest.approx(ws * 1000 * 10 / 2.0 / 1e6)
