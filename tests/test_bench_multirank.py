"""bench.py's multi-GPU path (replicas, no data-path collective): the timed
region is reduced to the slowest rank and the value counts every rank's work.
Run here as two gloo ranks on CPU."""
import os
import socket

import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [120.0, 200.0][rank]  # rank 1 is slower
    mx = bench.max_over_ranks(local_ms, dist, "cpu")
    value = bench.whole_job_value(10.0, 4, world, mx)
    out[rank] = (mx, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_max_and_whole_job_value():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        for r in range(2):
            mx, value = out[r]
            assert mx == 200.0
            assert abs(value - 2 * 10.0 * 4 / 0.2) < 1e-9


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.whole_job_value(1.0, 2, 1, 1000.0) == 2.0
