"""The multi-GPU form is replicas (no data-path collective): bench.py's
reduction of the timings over ranks and the whole-job value, on two CPU
processes with the gloo backend."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, ws, port, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    local = [100.0 + 50.0 * rank, 300.0 - 10.0 * rank]     # factor+solve ms, step ms
    fs, step = bench.max_over_ranks(local, torch.device("cpu"), ws)
    out[rank] = (fs, step, bench.replica_value(ws, 65536, 3, fs))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    ws = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(ws, _free_port(), out), nprocs=ws, join=True, start_method="spawn")
        res = dict(out)
    assert res[0] == res[1]
    fs, step, value = res[0]
    assert fs == 150.0 and step == 300.0
    assert value == pytest.approx(2 * 65536 * 3 / 0.150)


def test_one_process_is_the_identity():
    import bench
    assert bench.max_over_ranks([1.5, 2.5], None, 1) == [1.5, 2.5]
    assert bench.replica_value(1, 1000, 2, 500.0) == pytest.approx(4000.0)
