"""Batched instances, CUDA-graph replay and the schedule autotuner.

A batch of independent uneven-size Riemann problems advanced in the same
launches must give, instance by instance, exactly what each instance gives
alone (per-instance tau_n; rows never read another instance), under every
schedule (block size, graph replay) and in both precisions.
"""
import numpy as np
import pytest

import oracle as O
from gpu_common import rel_field_err, rel_field_err_l2, require_gpu
from paper_2007_00094_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


@pytest.fixture(scope="module")
def batch():
    parts = W.random_riemann_batch(n_instances=5, side_range=(5, 9), seed=4)
    mesh, off, U = W.concat_meshes([m for m, _ in parts], [u for _, u in parts])
    return parts, mesh, off, U


def _solver(mesh, **kw):
    from paper_2007_00094_gb300.idp import Solver
    return Solver(mesh, **kw)


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_equals_instances_alone(batch, precision):
    parts, mesh, off, U = batch
    s = _solver(mesh, precision=precision)
    s.set_instances(off)
    s.init_state(U)
    s.step(3)
    s.synchronize()
    out = s.get_state()
    t_batch, _ = s.instance_times()
    for k, (m, u) in enumerate(parts):
        a = _solver(m, precision=precision)
        a.init_state(u)
        a.step(3)
        a.synchronize()
        np.testing.assert_array_equal(out[:, off[k]:off[k + 1]], a.get_state())
        assert t_batch[k] == a.time()[0]
    assert len(set(t_batch)) > 1  # instances really took their own tau_n


def test_batch_matches_oracle(batch, n_threads):
    parts, mesh, off, U = batch
    s = _solver(mesh)
    s.set_instances(off)
    s.init_state(U)
    s.step(2)
    s.synchronize()
    out = s.get_state()
    for k, (m, u) in enumerate(parts):
        om = O.assemble(m)
        ref = u
        for _ in range(2):
            ref, _, st = O.ssprk3_step(om, ref, O.default_params(n_threads=n_threads))
            assert st == 0
        got = out[:, off[k]:off[k + 1]]
        assert rel_field_err_l2(got, ref).max() <= 1e-12
        assert rel_field_err(got, ref).max() <= 1e-11


@pytest.mark.parametrize("precision", [0, 1])
def test_schedules_and_graph_replay_are_bitwise_equal(batch, precision):
    """Per-step kernels and the persistent (one cooperative launch per
    euler_step) schedule, each with and without graph replay, at every
    block size, give bitwise the same states."""
    parts, mesh, off, U = batch
    outs = []
    for persistent in (False, True):
        for block in (64, 128, 256):
            for graph in (False, True):
                s = _solver(mesh, precision=precision)
                s.set_instances(off)
                s.set_schedule(block, graph, persistent)
                s.init_state(U)
                s.step(3)
                s.synchronize()
                outs.append(s.get_state())
                # per-step kernels: 7 per euler_step in FP64, 6 in FP32-mixed (its edge kernel
                # also forms the CFL bound); persistent: one per euler_step
                assert s.launch_count() == 3 * (3 if persistent else (21 if precision == 0 else 18))
    for o in outs[1:]:
        np.testing.assert_array_equal(o, outs[0])


@pytest.mark.parametrize("precision", [0, 1])
def test_persistent_schedule_on_a_large_mesh(precision):
    """More rows than co-resident threads: the persistent kernel's blocks loop
    over rows (grid-stride); results equal the per-step kernels bitwise."""
    mesh = W.vortex_mesh(48)
    U = W.bumpy_vortex_state(mesh)
    out = []
    for persistent in (False, True):
        s = _solver(mesh, precision=precision)
        s.set_schedule(256, False, persistent)
        s.init_state(U)
        s.step(2)
        s.synchronize()
        out.append(s.get_state())
    np.testing.assert_array_equal(out[0], out[1])


def test_grid_barrier_selftest_and_timeout(batch):
    """The persistent schedule's grid barrier: all blocks pass every round;
    with one block absent the other blocks' bounded waits run out, the call
    reports IDP_ERR_TIMEOUT and the context stays usable."""
    parts, mesh, off, U = batch
    s = _solver(mesh)
    st, passes = s.barrier_selftest(blocks=152, rounds=10)
    assert st == 0 and passes == 1520
    st, passes = s.barrier_selftest(blocks=152, rounds=10, skip_block0=True, spin_limit=1000)
    assert st == 8  # IDP_ERR_TIMEOUT
    assert passes == 0
    s.set_instances(off)
    s.init_state(U)
    s.step(1)
    s.synchronize()
    assert np.all(np.isfinite(s.get_state()))


def test_instances_must_not_share_entries(batch):
    from paper_2007_00094_gb300.idp import IdpError
    parts, mesh, off, U = batch
    s = _solver(mesh)
    bad = off.copy()
    bad[1] += 3  # splits the first cube
    with pytest.raises(IdpError) as e:
        s.set_instances(bad)
    assert e.value.status == 1


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_with_relaxed_bounds_equals_instances_alone(batch, precision):
    """With bound relaxation r_i = (m_i / |Omega_k|)^(1/2) each instance uses
    its own volume |Omega_k|: the batch equals each instance alone, bitwise."""
    parts, mesh, off, U = batch
    s = _solver(mesh, precision=precision, relax=1)
    s.set_instances(off)
    s.init_state(U)
    s.step(2)
    s.synchronize()
    out = s.get_state()
    for k, (m, u) in enumerate(parts):
        a = _solver(m, precision=precision, relax=1)
        a.init_state(u)
        a.step(2)
        a.synchronize()
        np.testing.assert_array_equal(out[:, off[k]:off[k + 1]], a.get_state())


@pytest.mark.parametrize("precision", [0, 1])
def test_2d_batch_equals_instances_alone_and_matches_oracle(precision, n_threads):
    """A batch of 2D Riemann problems (Q1 quadrilaterals): bitwise equal to each
    instance alone, and (FP64) within the parity tolerance of the oracle."""
    parts = W.random_riemann_batch_2d(n_instances=4, side_range=(6, 15), seed=6)
    mesh, off, U = W.concat_meshes([m for m, _ in parts], [u for _, u in parts])
    s = _solver(mesh, precision=precision)
    s.set_instances(off)
    s.init_state(U)
    s.step(2)
    s.synchronize()
    out = s.get_state()
    assert not out[3].any()
    for k, (m, u) in enumerate(parts):
        a = _solver(m, precision=precision)
        a.init_state(u)
        a.step(2)
        a.synchronize()
        got = out[:, off[k]:off[k + 1]]
        np.testing.assert_array_equal(got, a.get_state())
        if precision == 0:
            om = O.assemble(m)
            ref = u
            for _ in range(2):
                ref, _, st = O.ssprk3_step(om, ref, O.default_params(n_threads=n_threads))
                assert st == 0
            assert rel_field_err_l2(got, ref).max() <= 1e-12
            assert rel_field_err(got, ref).max() <= 1e-11
