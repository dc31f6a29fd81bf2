"""The multi-GPU path of bench.py is replicas: each rank decomposes its own
copy of the workload and the ranks only reduce their times and work. This is
checked here with two gloo ranks on the CPU (no GPU)."""
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


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, units = bench.job_totals(10.0 + 5.0 * rank, 1000 * (rank + 1))
    out[rank] = (ms, units)
    # each rank sees the same replica workload (same seed => same graph)
    import graphgen as gg
    g = gg.rmat_graph(10, 8, gg.SEED_BASE + 3)
    h = torch.tensor([int(g.col_idx.sum()), g.arcs], dtype=torch.int64)
    allh = [torch.zeros_like(h) for _ in range(world)]
    dist.all_gather(allh, h)
    out[world + rank] = all(torch.equal(allh[0], x) for x in allh)
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_time_and_work():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        # slowest rank's time, all ranks' work
        assert out[0] == (15.0, 3000) and out[1] == (15.0, 3000)
        assert out[2] and out[3]


def test_single_process_is_identity():
    import bench
    if dist.is_initialized():
        pytest.skip("a process group is active")
    assert bench.job_totals(12.5, 77) == (12.5, 77)
