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
