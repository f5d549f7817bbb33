"""The multi-rank (N > 1) path of bench.py on CPU: world_size 2 over gloo.
Each rank advances its own replica (no data-path collective); the whole-job
rate is all ranks' units over the slowest rank's time."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert bench._dist() == (world, rank, rank)
        local_ms = 100.0 + 50.0 * rank  # rank 1 is the slow one
        ms_max, rate = bench.job_rate(local_ms, 3.0e6, dist)
        out[rank] = (ms_max, rate)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_job_rate_takes_max_over_two_gloo_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as manager:
        out = manager.dict()
        procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(world):
        ms_max, rate = res[r]
        assert ms_max == 150.0
        assert abs(rate - 2 * 3.0e6 / 0.150) <= 1e-9 * rate


def test_job_rate_single_process():
    sys.path.insert(0, ROOT)
    import bench
    ms, rate = bench.job_rate(200.0, 1.0e6)
    assert ms == 200.0 and abs(rate - 5.0e6) < 1e-6
