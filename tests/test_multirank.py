"""Multi-rank paths on CPU, world_size 2 over gloo: bench.py's N > 1 run,
where each rank advances its own replica (no data-path collective) and the
whole-job rate is all ranks' units over the slowest rank's time; and the
sharded stage's halo exchange between ranks (shard.HaloExchange over a
ShardPlan: ghosts receive their owners' node and entry values, tau is the
minimum over ranks)."""
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


def _halo_rank_main(rank, world, port, out):
    """One shard per rank: ghosts start as NaN and must hold the owners'
    values after the exchanges; the CFL bound is the minimum over ranks."""
    sys.path.insert(0, ROOT)
    import numpy as np

    from paper_2007_00094_gb300 import workloads as W
    from paper_2007_00094_gb300.idp import ShardPlan
    from paper_2007_00094_gb300.shard import HaloExchange
    from test_shard_plan import _pattern

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mesh = W.forward_step_mesh(m=10, jitter=0.2, seed=2007)
        rowptr, col = _pattern(mesh)
        n, nnz = len(rowptr) - 1, len(col)
        plan = ShardPlan(rowptr, col, world)
        # the same global fields on every rank (seeded), standing in for R_j and l_ij
        rng = np.random.default_rng(11)
        X = rng.standard_normal((5, n))
        Y = rng.random(nnz)
        cand = rng.random(n) + 0.5
        nodes = plan.nodes(rank)
        nl, lo, hi, el = plan.info(rank)
        _, lcol, entry = plan.csr(rank)
        lrp = plan.csr(rank)[0]
        lrows = np.repeat(np.arange(nl), np.diff(lrp))
        Xl = torch.full((5, nl), float("nan"), dtype=torch.float64)
        Xl[:, lo:hi] = torch.from_numpy(X[:, nodes[lo:hi]])
        Yl = torch.full((el,), float("nan"), dtype=torch.float64)
        own = (lrows >= lo) & (lrows < hi)
        Yl[torch.from_numpy(own)] = torch.from_numpy(Y[entry[own]])
        ex = HaloExchange(plan, rank)
        ex.exchange_nodes(Xl)
        ex.exchange_entries(Yl)
        node_ok = bool(np.array_equal(Xl.numpy(), X[:, nodes]))
        # entries of ghost rows into own rows now hold the owners' values
        need = (~own) & (lcol >= lo) & (lcol < hi)
        entry_ok = bool(np.array_equal(Yl.numpy()[need], Y[entry[need]])) and bool(need.any())
        t = torch.tensor([cand[nodes[lo:hi]].min()], dtype=torch.float64)
        ex.min_allreduce(t)
        out[rank] = (node_ok, entry_ok, float(t.item()), float(cand.min()))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_halo_exchange_over_two_gloo_ranks():
    pytest.importorskip("paper_2007_00094_gb300.idp")
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as manager:
        out = manager.dict()
        procs = [ctx.Process(target=_halo_rank_main, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(world):
        node_ok, entry_ok, tau, tau_ref = res[r]
        assert node_ok and entry_ok, r
        assert tau == tau_ref
