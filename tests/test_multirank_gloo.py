"""The multi-GPU path of the benchmark, run as world-size-2 gloo ranks on CPU:
every rank works on its own CPI (a different sub-seed, no data exchange), the
job time is the slowest rank's, and the value counts every rank's cells."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from paper_2203_06233_gb300 import synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    spec = bench.workload_spec(rank)
    cube = synth.make_cube(spec)
    local_ms = 10.0 * (rank + 1)                      # rank 1 is the slow one
    total, value = bench.aggregate(local_ms, spec.cells, world, torch.device("cpu"))
    checksum = torch.tensor([float(np.abs(cube).sum())], dtype=torch.float64)
    sums = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(sums, checksum)
    q.put((rank, spec.sub, total, value, [float(x) for x in sums]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_weak_scaling_aggregate():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    cells = synth.standard_cpi().cells
    for rank, sub, total, value, sums in res:
        assert sub == rank                              # each rank its own CPI
        assert total == pytest.approx(20.0)             # the slowest rank's time
        assert value == pytest.approx(world * cells / 20e-3)
        assert sums[0] != sums[1]                       # different data on each rank
