"""Rotation invariance of the oracle's stage on uniform periodic grids.

The Euler equations commute with rotations, and on a uniform periodic grid
the Q1 scheme does too: a cyclic permutation of the axes in 3D and a quarter
turn in 2D map the mesh onto itself.  One euler_step of the rotated state
must equal the rotated euler_step of the state, up to rounding (row sums run
in another order).  A transposed operand, a swapped component or an index
mix-up in the assembly, the fluxes, the wavespeed, the indicator or the
limiter breaks this.
"""
import numpy as np
import pytest

import oracle as O
from paper_2007_00094_gb300 import workloads as W


def _state(x, seed):
    rng = np.random.default_rng(seed)
    k = rng.uniform(1.0, 3.0, size=(4, x.shape[1]))
    ph = rng.uniform(0.0, 2 * np.pi, size=4)
    wave = [np.sin(2 * np.pi * (x @ k[q].round()) + ph[q]) for q in range(4)]
    rho = 1.0 + 0.3 * wave[0] + 0.5 * (x[:, 0] > 0.5)  # a jump for the limiter
    u = np.stack([0.4 * wave[1], 0.3 * wave[2], 0.2 * wave[3]])
    p = 1.0 + 0.2 * wave[1] * wave[2] + 0.8 * (x[:, 1] > 0.4)
    return rho, u, p


def test_cyclic_axis_permutation_3d(n_threads):
    n = 8
    mesh = W.vortex_mesh(n)
    om = O.assemble(mesh)
    ii, jj, kk = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    ii, jj, kk = (a.transpose(2, 1, 0).ravel() for a in (ii, jj, kk))
    rho, u, p = _state(mesh.x, 1)
    U = W.primitive_to_conserved(rho, u, p)
    # T(x, y, z) = (y, z, x): node (i, j, k) of the rotated field holds old node (k, i, j), m' = (m_y, m_z, m_x)
    src = kk + n * (ii + n * jj)

    def rot(V):
        R = V[:, src].copy()
        R[1:4] = V[[2, 3, 1]][:, src]
        return R

    prm = O.default_params(n_threads=n_threads)
    E, tau, st, _ = O.euler_step(om, U, params=prm)
    Er, taur, str_, _ = O.euler_step(om, rot(U), params=prm)
    assert st == 0 and str_ == 0
    assert abs(tau - taur) <= 1e-14 * tau
    scale = np.abs(E).max(axis=1, keepdims=True)
    assert (np.abs(Er - rot(E)) / scale).max() <= 1e-12


def test_quarter_turn_2d(n_threads):
    n = 16
    mesh = W.vortex_mesh_2d(n)
    om = O.assemble(mesh)
    jj, ii = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    ii, jj = ii.ravel(), jj.ravel()
    rho, u, p = _state(mesh.x[:, :2], 2)
    u[2] = 0.0
    U = W.primitive_to_conserved(rho, u, p)
    # T(x, y) = (-y, x): node (i, j) of the rotated field holds old node (j, -i mod n), m' = (-m_y, m_x)
    src = jj + n * ((-ii) % n)

    def rot(V):
        R = V[:, src].copy()
        R[1] = -V[2, src]
        R[2] = V[1, src]
        return R

    prm = O.default_params(n_threads=n_threads)
    E, tau, st, _ = O.euler_step(om, U, params=prm)
    Er, taur, str_, _ = O.euler_step(om, rot(U), params=prm)
    assert st == 0 and str_ == 0
    assert abs(tau - taur) <= 1e-14 * tau
    scale = np.abs(E).max()
    assert np.abs(Er - rot(E)).max() <= 1e-12 * scale
    assert not Er[3].any()
