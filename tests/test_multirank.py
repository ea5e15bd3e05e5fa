"""The benchmark's multi-GPU logic on CPU ranks (gloo, world size 2): each
rank gets its own block, the step time is the maximum over ranks, and the
job's throughput counts every rank's cells. There is no data-path
collective: cells and masking statistics are per block."""
import os
import socket

import pytest

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cfg, _ = bench.workload("small", rank)
    ms = 10.0 + 5.0 * rank                       # the second rank is slower
    ms_max = bench.max_over_ranks(ms, dist)
    value = bench.job_throughput(cfg.n_cells, world, ms_max)
    out.put((rank, cfg.seed, ms_max, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, m0, v0), (r1, s1, m1, v1) = res
    assert s0 != s1                               # independent blocks
    assert m0 == m1 == 15.0                       # max over ranks
    cells = bench.workload("small", 0)[0].n_cells
    assert v0 == v1 == pytest.approx(2 * cells / 0.015)


def test_single_process_is_identity():
    assert bench.max_over_ranks(3.5, None) == 3.5
    assert bench.job_throughput(100, 1, 1000.0) == 100.0
