"""The sharded stage (Sec. 4.1, Fig. 1-2) on one GPU: the rows split into
contiguous ranges, one context per shard with one ghost layer, halo
exchanges of alpha, R, l (twice) and U plus a min-reduction of the CFL
bound between the stage's phases.  Every own row computes what the
unsharded stage computes, in the same order, so states, time and tau_n must
be bitwise equal to idp_step on the same matrices; one step is also checked
against the FP64 oracle at the parity tolerance of the unsharded stage."""
import numpy as np
import pytest

import oracle as O
from gpu_common import rel_field_err, require_gpu
from paper_2007_00094_gb300 import workloads as W
from test_gpu_parity import _mesh

pytestmark = pytest.mark.gpu


def _sparsity(mesh):
    from paper_2007_00094_gb300.idp import Solver

    s = Solver(mesh)
    rowptr, col, mij, cij, mi = s.matrices()
    s.close()
    return dict(rowptr=rowptr, col=col, mij=mij, cij=cij, mi=mi, bc=mesh.bc, inflow=mesh.inflow)


def _run_both(mesh, U, n_shards, steps, row_begin=None, mi=True, precision=0):
    from paper_2007_00094_gb300.idp import ShardedSolver, Solver

    sp = _sparsity(mesh)
    ref = Solver(sparsity=sp, precision=precision)
    ref.init_state(U)
    ref.step(steps)
    ref.synchronize()
    out_ref, t_ref = ref.get_state(), ref.time()
    ref.close()
    if not mi:
        sp = dict(sp, mi=None)
    sh = ShardedSolver(sp, n_shards=n_shards, row_begin=row_begin, precision=precision)
    sh.init_state(U)
    sh.step(steps)
    sh.synchronize()
    out, t = sh.get_state(), sh.time()
    halo = sh.halo_size()
    sh.close()
    return out, t, out_ref, t_ref, halo


@pytest.mark.parametrize("name", ["vortex17", "ffs10", "wallbox_jitter", "sod_jitter", "ffs2d_10",
                                  "wallrect_jitter"])
@pytest.mark.parametrize("n_shards", [2, 3])
@pytest.mark.parametrize("precision", [0, 1])
def test_sharded_bitwise_equals_unsharded(name, n_shards, precision):
    """FP64 and FP32-mixed (whose shards exchange FP32 alpha, R and l and use
    the whole mesh's scale for the FP32 copies of c_ij)."""
    require_gpu()
    mesh, U = _mesh(name)
    out, t, out_ref, t_ref, halo = _run_both(mesh, U, n_shards, steps=3, precision=precision)
    assert halo[0] > 0 and halo[1] > 0
    assert t == t_ref, (t, t_ref)
    assert np.array_equal(out, out_ref), float(np.abs(out - out_ref).max())


@pytest.mark.parametrize("precision", [0, 1])
def test_sharded_uneven_ranges_and_row_sum_masses(precision):
    require_gpu()
    mesh, U = _mesh("ffs10")
    n = mesh.n_nodes
    # four shards of unequal size, one of them a single slice; lumped masses
    # formed by the group as row sums of m_ij (no mi given)
    rb = [0, 37, 37 + 32, n // 2 + 5, n]
    out, t, out_ref, t_ref, _ = _run_both(mesh, U, 4, steps=2, row_begin=rb, mi=False, precision=precision)
    assert t == t_ref
    assert np.array_equal(out, out_ref)


def test_sharded_mixed_on_a_structured_grid_keeps_table_and_patterns():
    """On a uniform grid the shards' FP32-mixed contexts still find the entry
    table and row patterns (ghost rows add patterns of their own) and stay
    bitwise equal to the unsharded stage."""
    require_gpu()
    mesh = W.sod_cube_mesh(24)
    U = W.sod_state(mesh)
    out, t, out_ref, t_ref, _ = _run_both(mesh, U, 3, steps=3, precision=1)
    assert t == t_ref
    assert np.array_equal(out, out_ref)


def test_sharded_matches_the_oracle():
    require_gpu()
    from paper_2007_00094_gb300.idp import ShardedSolver

    for name in ("ffs10", "sod_jitter"):
        mesh, U = _mesh(name)
        sh = ShardedSolver(_sparsity(mesh), n_shards=3)
        sh.init_state(U)
        sh.step(1)
        sh.synchronize()
        out = sh.get_state()
        sh.close()
        ref, tau, st = O.ssprk3_step(O.assemble(mesh), U)
        assert st == 0
        err = rel_field_err(out, ref)
        assert err.max() <= 1e-12, (name, err)


def test_sharded_rejects_unsupported_configs():
    require_gpu()
    from paper_2007_00094_gb300.idp import IdpError, ShardedSolver

    mesh, _ = _mesh("tiny3")
    sp = _sparsity(mesh)
    for kw in (dict(relax=1), dict(renumber=1), dict(precision=2)):
        with pytest.raises(IdpError):
            ShardedSolver(sp, n_shards=2, **kw)


def test_sharded_rejects_non_admissible_state():
    require_gpu()
    from paper_2007_00094_gb300.idp import IdpError, ShardedSolver

    mesh, U = _mesh("vortex17")
    sh = ShardedSolver(_sparsity(mesh), n_shards=2)
    Ub = U.copy()
    Ub[0, mesh.n_nodes - 3] = -1.0  # a row of the second shard
    with pytest.raises(IdpError):
        sh.init_state(Ub)
    sh.close()


@pytest.mark.parametrize("n_shards", [1, 2, 3, 5])
def test_sharded_degenerate_partitions(n_shards):
    """Edge cases of the partition: one shard (no links: the plain stage in
    phases), and the 3^3 periodic vortex, where every node neighbours every
    other through the periodic seams, so each shard holds nearly the whole
    mesh as ghosts and exchanges with every other shard."""
    require_gpu()
    mesh, U = _mesh("tiny3")
    out, t, out_ref, t_ref, halo = _run_both(mesh, U, n_shards, steps=2)
    assert t == t_ref
    assert np.array_equal(out, out_ref)
    if n_shards == 1:
        assert halo[:2] == (0, 0)
