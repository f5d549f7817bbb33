"""Functionals J(U) of a state, with their gradients dJ/dU, as seeds for the
discrete adjoint (``Solver.adjoint_backward`` / ``idp.rollout``).

States are (5, N) conserved variables (rho, m_x, m_y, m_z, E) with
gamma = 7/5, p = (gamma - 1)(E - |m|^2/(2 rho)) (Sec. 2).
"""
from __future__ import annotations

import numpy as np

GAMMA = 1.4


class BoxPressure:
    """J(U) = sum over nodes x_i in [lo, hi]^3 of m_i p_i: the lumped-mass
    quadrature of the pressure integral over the box.  ``mi`` are the lumped
    masses m_i (e.g. from ``Solver.matrices()``), ``x`` the node positions."""

    def __init__(self, x, mi, lo=0.4, hi=0.6):
        inside = np.all((x >= lo) & (x <= hi), axis=1)
        self.w = np.where(inside, np.asarray(mi, dtype=np.float64), 0.0)
        self.n_inside = int(inside.sum())

    def __call__(self, U):
        eps = U[4] - 0.5 * (U[1] ** 2 + U[2] ** 2 + U[3] ** 2) / U[0]
        return float((self.w * (GAMMA - 1.0) * eps).sum())

    def gradient(self, U):
        """dJ/dU: m_i (gamma - 1) (|v|^2/2, -v, 1) inside the box, 0 elsewhere."""
        v = U[1:4] / U[0]
        g = np.empty_like(U)
        g[0] = self.w * (GAMMA - 1.0) * 0.5 * (v * v).sum(axis=0)
        g[1:4] = -self.w * (GAMMA - 1.0) * v
        g[4] = self.w * (GAMMA - 1.0)
        return g
