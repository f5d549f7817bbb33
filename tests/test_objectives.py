"""The adjoint seeds of paper_2007_00094_gb300.objectives against central
differences (host only)."""
import numpy as np

from paper_2007_00094_gb300 import workloads as W
from paper_2007_00094_gb300.objectives import BoxPressure


def test_box_pressure_gradient_and_value():
    mesh = W.vortex_mesh(9)
    U = W.bumpy_vortex_state(mesh)
    mi = np.random.default_rng(0).uniform(0.5, 1.5, mesh.n_nodes)
    J = BoxPressure(mesh.x, mi)
    assert J.n_inside > 0
    rho, u, p = W.vortex_primitive(mesh.x)
    inside = np.all((mesh.x >= 0.4) & (mesh.x <= 0.6), axis=1)
    # value: the lumped quadrature of p over the box (bumps change rho only)
    assert abs(J(U) - float((mi * p)[inside].sum())) <= 1e-12 * abs(J(U))
    g = J.gradient(U)
    assert np.all(g[:, ~inside] == 0.0)
    rng = np.random.default_rng(1)
    for _ in range(4):
        v = rng.standard_normal(U.shape) * np.abs(U)
        eps = 1e-6
        fd = (J(U + eps * v) - J(U - eps * v)) / (2 * eps)
        assert abs(fd - float((g * v).sum())) <= 1e-7 * abs(fd)
