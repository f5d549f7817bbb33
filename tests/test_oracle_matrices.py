"""Pins for the oracle's Q1 assembly (Sec. 3.1 eq. "matrices").

The oracle's m_ij, c_ij, m_i are checked against closed forms on uniform
grids and against identities that hold on any mesh: partition of unity,
reproduction of linear functions, and the boundary identity
c_ij + c_ji = int_{dOmega} phi_i phi_j n.
"""
import numpy as np
import pytest

import oracle as O
from paper_2007_00094_gb300 import workloads as W

from helpers import csr_rows, transpose_index


def _offset(mesh, om, i, j):
    shape = np.array(mesh.meta["shape"])
    gi = np.array([i % shape[0], (i // shape[0]) % shape[1], i // (shape[0] * shape[1])])
    gj = np.array([j % shape[0], (j // shape[0]) % shape[1], j // (shape[0] * shape[1])])
    d = gj - gi
    return (d + shape // 2) % shape - shape // 2  # minimum image on the periodic grid


def test_uniform_periodic_closed_forms():
    n = 6
    mesh = W.vortex_mesh(n)
    om = O.assemble(mesh)
    h = 1.0 / n
    M1 = {0: 2 * h / 3, 1: h / 6, -1: h / 6}
    C1 = {0: 0.0, 1: 0.5, -1: -0.5}
    assert om.nnz == 27 * om.n
    np.testing.assert_allclose(om.mi, h ** 3, rtol=1e-14)
    for i in [0, 7, 100, om.n - 1]:
        cols, m, c = om.dense_row(i)
        for q, j in enumerate(cols):
            dx, dy, dz = _offset(mesh, om, i, j)
            assert abs(m[q] - M1[dx] * M1[dy] * M1[dz]) < 1e-15
            expect = [C1[dx] * M1[dy] * M1[dz], M1[dx] * C1[dy] * M1[dz], M1[dx] * M1[dy] * C1[dz]]
            np.testing.assert_allclose(c[:, q], expect, atol=1e-16)
    # face, edge, corner neighbours: 2h^2/9, h^2/18, h^2/72 per component
    cols, m, c = om.dense_row(0)
    mags = sorted(set(np.round(np.abs(c[np.abs(c) > 1e-12 * h ** 2]) / h ** 2, 12)))
    np.testing.assert_allclose(mags, [1 / 72, 1 / 18, 2 / 9], rtol=1e-10)
    # sum_j |c_ij| (Euclidean) = (6 * 2/9 + 12 * sqrt(2)/18 + 8 * sqrt(3)/72) h^2
    s = np.sqrt((c ** 2).sum(axis=0)).sum()
    assert abs(s - (6 * 2 / 9 + 12 * np.sqrt(2) / 18 + 8 * np.sqrt(3) / 72) * h ** 2) < 1e-15


@pytest.mark.parametrize("name", ["wallbox", "periodic_jitter", "ffs"])
def test_identities_any_mesh(name):
    if name == "wallbox":
        mesh = W.box_mesh((7, 5, 6), hi=(1.3, 0.9, 1.1), periodic=(False, False, False), jitter=0.25, seed=3)
    elif name == "periodic_jitter":
        mesh = W.box_mesh((6, 5, 7), periodic=(True, True, True), jitter=0.25, seed=4)
    else:
        mesh = W.forward_step_mesh(m=10, jitter=0.2, seed=2007)
    om = O.assemble(mesh)
    rows = csr_rows(om)
    kT = transpose_index(om)
    scale_m = om.mi.max()
    scale_c = np.abs(om.cij).max()
    # partition of unity: sum_j m_ij = m_i, sum_j c_ij = 0; sum_i m_i = |Omega|
    np.testing.assert_allclose(np.bincount(rows, om.mij), om.mi, atol=1e-14 * scale_m)
    for d in range(3):
        assert np.abs(np.bincount(rows, om.cij[d], minlength=om.n)).max() < 1e-14 * scale_c
    assert abs(om.mi.sum() - mesh.volume) < 1e-12 * mesh.volume
    # symmetry of the consistent mass
    np.testing.assert_array_equal(om.mij, om.mij[kT])
    # reproduction of linear functions: sum_j c_ij (a . x_j) = m_i a
    if not any(mesh.periodic):
        rng = np.random.default_rng(0)
        a = rng.normal(size=3)
        lin = mesh.x @ a
        for d in range(3):
            got = np.bincount(rows, om.cij[d] * lin[om.col], minlength=om.n)
            np.testing.assert_allclose(got, om.mi * a[d], atol=1e-13 * scale_m * np.abs(a).max())
    # c_ij + c_ji vanishes away from the boundary, sum_i sum_j c_ij = int_dOmega n = 0
    skew = om.cij + om.cij[:, kT]
    interior = mesh.bc[rows] == 0
    interior &= mesh.bc[om.col] == 0
    if name == "ffs":
        on_bnd = np.zeros(om.n, dtype=bool)
        on_bnd[(mesh.x[:, 0] < 1e-12) | (mesh.x[:, 0] > 3 - 1e-12)] = True
        interior &= ~on_bnd[rows] & ~on_bnd[om.col]
    assert np.abs(skew[:, interior]).max() < 1e-14 * scale_c
    assert np.abs(om.cij.sum(axis=1)).max() < 1e-12 * scale_c


def test_boundary_identity_wall_box():
    """sum_j c_ji = int_dOmega phi_i n: on an axis-aligned box, node i on the
    face x = 0 (away from edges) gets (-h^2, 0, 0) on a uniform grid."""
    n = 5
    mesh = W.box_mesh((n, n, n), periodic=(False, False, False))
    om = O.assemble(mesh)
    kT = transpose_index(om)
    rows = csr_rows(om)
    h = 1.0 / (n - 1)
    col_sum = np.stack([np.bincount(rows, om.cij[d][kT], minlength=om.n) for d in range(3)])
    for i in range(om.n):
        gi = (i % n, (i // n) % n, i // (n * n))
        expect = np.zeros(3)
        for d in range(3):
            face_area = 1.0
            for e in range(3):
                if e != d:
                    face_area *= h / 2 if gi[e] in (0, n - 1) else h
            if gi[d] == 0:
                expect[d] = -face_area
            elif gi[d] == n - 1:
                expect[d] = face_area
        np.testing.assert_allclose(col_sum[:, i], expect, atol=1e-15)


def test_forward_step_full_size_counts():
    """The h = 1/120 channel has the node count quoted for the workload."""
    m = 120
    nx, ny, nz = 3 * m + 1, m + 1, m // 2 + 1
    removed = (nx - 1 - (6 * m) // 10) * ((2 * m) // 10) * nz
    assert nx * ny * nz - removed == 2_242_909
    small = W.forward_step_mesh(m=10)
    nx, ny, nz = 31, 11, 6
    assert small.n_nodes == nx * ny * nz - (30 - 6) * 2 * nz


def test_sparsity_counts():
    mesh = W.box_mesh((4, 5, 6), periodic=(False, False, False))
    om = O.assemble(mesh)
    counts = np.diff(om.rowptr)
    for i in range(om.n):
        g = (i % 4, (i // 4) % 5, i // 20)
        expect = 1
        for gi, n in zip(g, (4, 5, 6)):
            expect *= 2 if gi in (0, n - 1) else 3
        assert counts[i] == expect
    # columns sorted and unique
    for i in range(om.n):
        c = om.col[om.rowptr[i]:om.rowptr[i + 1]]
        assert (np.diff(c) > 0).all()
