"""Seeded input generators: shapes, flags and the batch concatenation."""
import numpy as np

from paper_2007_00094_gb300 import workloads as W


def test_concat_meshes_offsets_and_cells():
    parts = [W.box_mesh((n, n, n), periodic=(False, False, False)) for n in (3, 4, 5)]
    states = [W.uniform_state(m, rho=1.0 + k) for k, m in enumerate(parts)]
    mesh, off, U = W.concat_meshes(parts, states)
    assert list(off) == [0, 27, 27 + 64, 27 + 64 + 125]
    assert mesh.n_nodes == off[-1] and U.shape == (5, off[-1])
    for k, m in enumerate(parts):
        block = mesh.cells[sum(p.n_cells for p in parts[:k]):sum(p.n_cells for p in parts[:k + 1])]
        assert block.min() >= off[k] and block.max() < off[k + 1]
        np.testing.assert_array_equal(block - off[k], m.cells)
        assert np.all(U[0, off[k]:off[k + 1]] == 1.0 + k)


def test_random_riemann_batch_is_seeded():
    a = W.random_riemann_batch(n_instances=4, side_range=(4, 6), seed=4)
    b = W.random_riemann_batch(n_instances=4, side_range=(4, 6), seed=4)
    for (ma, ua), (mb, ub) in zip(a, b):
        assert ma.n_nodes == mb.n_nodes
        np.testing.assert_array_equal(ua, ub)
        rho = ua[0]
        assert rho.min() >= 0.1 and rho.max() <= 2.0


def test_forward_step_flags():
    m = W.forward_step_mesh(m=10, jitter=0.2, seed=2007)
    x = m.x
    assert np.all(m.bc[np.isclose(x[:, 0], 0.0)] == W.BC_INFLOW)
    top = np.isclose(x[:, 1], 1.0) & (x[:, 0] > 1e-12)
    assert np.all(m.bc[top] & W.BC_SLIP_Y)
    face = np.isclose(x[:, 0], 0.6) & (x[:, 1] < 0.2 - 1e-12) & (x[:, 1] > 1e-12)
    assert face.any() and np.all(m.bc[face] & W.BC_SLIP_X)
    interior = m.bc == 0
    assert interior.any()


def test_2d_generators():
    """Quadrilateral meshes: counts of the 2D step (h = 1/1000 gives the
    2,524,001 nodes quoted for the benchmark), unwrapped periodic vertices,
    zero z coordinates, and the slip/inflow flags of the channel."""
    nx, ny, m = 3001, 1001, 1000
    assert nx * ny - (nx - 1 - 600) * 200 == 2_524_001
    small = W.forward_step_mesh_2d(m=20, jitter=0.2, seed=1)
    assert small.dim == 2 and small.n_nodes == 61 * 21 - (60 - 12) * 4
    assert small.n_cells == 60 * 20 - 48 * 4
    assert not small.x[:, 2].any() and not small.cell_xyz[:, :, 2].any()
    inflow = small.x[:, 0] == 0.0
    assert (small.bc[inflow] == W.BC_INFLOW).all()
    step_top = (np.abs(small.x[:, 1] - 0.2) < 1e-12) & (small.x[:, 0] > 0.6 + 1e-12)
    assert (small.bc[step_top] & W.BC_SLIP_Y).all()
    per = W.rect_mesh((5, 4), periodic=(True, True))
    # every cell is a positively oriented unit-spaced square once unwrapped
    e1 = per.cell_xyz[:, 1, :2] - per.cell_xyz[:, 0, :2]
    e2 = per.cell_xyz[:, 2, :2] - per.cell_xyz[:, 0, :2]
    np.testing.assert_allclose(e1, [[0.2, 0.0]] * per.n_cells, atol=1e-15)
    np.testing.assert_allclose(e2, [[0.0, 0.25]] * per.n_cells, atol=1e-15)
    batch = W.random_riemann_batch_2d(n_instances=3, side_range=(5, 9), seed=2)
    assert all(mesh.dim == 2 and not U[3].any() for mesh, U in batch)
