"""Test-side state functions (Sec. 2) used to check invariants independently."""
import numpy as np

GAMMA = 1.4


def rho_eps(U):
    return U[0] * U[4] - 0.5 * (U[1] ** 2 + U[2] ** 2 + U[3] ** 2)


def internal_energy(U):
    return U[4] - 0.5 * (U[1] ** 2 + U[2] ** 2 + U[3] ** 2) / U[0]


def pressure(U, gamma=GAMMA):
    return (gamma - 1.0) * internal_energy(U)


def specific_entropy(U, gamma=GAMMA):
    return internal_energy(U) * U[0] ** (-gamma)


def primitive(U, gamma=GAMMA):
    rho = U[0]
    u = U[1:4] / rho
    return rho, u, pressure(U, gamma)


def csr_rows(om):
    """Row index of every CSR entry."""
    return np.repeat(np.arange(om.n), np.diff(om.rowptr))


def transpose_index(om):
    """Position of entry (j, i) for every entry (i, j)."""
    rows = csr_rows(om)
    key = rows * om.n + om.col
    keyT = om.col * om.n + rows
    order = np.argsort(key)
    pos = np.searchsorted(key[order], keyT)
    return order[pos]


def flux_dot(U, c, gamma=GAMMA):
    """f(U) . c for states U (5, m) and vectors c (3, m), eq. (flux)."""
    rho, m, E = U[0], U[1:4], U[4]
    v = m / rho
    p = pressure(U, gamma)
    mc = (m * c).sum(axis=0)
    out = np.empty_like(U)
    out[0] = mc
    out[1:4] = v * mc + p * c
    out[4] = (E + p) * (v * c).sum(axis=0)
    return out
