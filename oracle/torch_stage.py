"""Differentiable FP64 CPU restatement of one euler_step (Alg. 1) and SSP-RK3.

TEST INFRASTRUCTURE ONLY (reference gradient for the GPU adjoint).  The same
method as oracle/idp_oracle.c, written with plain PyTorch CPU tensor
operations over all stencil entries at once instead of loops, so that
torch.autograd differentiates the computation as performed: every max, min,
clamp and limiter branch routes the gradient to the branch the forward pass
took.  Its forward values are pinned to the C oracle (tests/test_oracle_torch.py).

Readings follow the C oracle (A1-A28 of the design notes); sections refer to
Maier & Kronbichler, arXiv:2007.00094.
"""
from __future__ import annotations

import numpy as np
import torch

GAMMA = 1.4
NF = 5


def _where(c, a, b):
    return torch.where(c, a, b)


def _safe(x, ok, fill=1.0):
    """x where ok, else a harmless value (keeps unused branches finite)."""
    return torch.where(ok, x, torch.full_like(x, fill))


class TorchMesh:
    """CSR matrices of an oracle.OracleMesh as tensors, plus entry bookkeeping."""

    def __init__(self, om):
        self.n = om.n
        rp = torch.as_tensor(om.rowptr)
        self.rows = torch.repeat_interleave(torch.arange(om.n), rp[1:] - rp[:-1])
        self.col = torch.as_tensor(om.col)
        key = self.rows * om.n + self.col
        keyT = self.col * om.n + self.rows
        order = torch.argsort(key)
        self.kT = order[torch.searchsorted(key[order], keyT)]
        self.diag = self.rows == self.col
        self.off = ~self.diag
        self.c = torch.as_tensor(om.cij)  # (3, nnz)
        self.cT = self.c[:, self.kT]
        self.mij = torch.as_tensor(om.mij)
        self.mi = torch.as_tensor(om.mi)
        self.card = (rp[1:] - rp[:-1]).to(torch.float64)
        self.lam = 1.0 / (self.card - 1.0)
        self.bc = torch.as_tensor(om.bc)
        self.inflow = torch.as_tensor(om.inflow)

    def row_sum(self, v):
        out = torch.zeros(v.shape[:-1] + (self.n,), dtype=v.dtype)
        return out.index_add(-1, self.rows, v)


def internal_energy(U):
    return U[4] - (U[1] ** 2 + U[2] ** 2 + U[3] ** 2) / (2.0 * U[0])


def pressure(U):
    return (GAMMA - 1.0) * internal_energy(U)


def specific_entropy(U):
    return internal_energy(U) * U[0] ** (-GAMMA)


def flux_dot(U, c):
    """f(U) . c (eq. flux) for states (5, m) and vectors (3, m)."""
    rho, m, E = U[0], U[1:4], U[4]
    v = m / rho
    p = pressure(U)
    out = [(m * c).sum(0)]
    for r in range(3):
        out.append((v[r] * m * c).sum(0) + p * c[r])
    out.append(((v * c).sum(0)) * (E + p))
    return torch.stack(out)


def lambda_max(n, Ui, Uj):
    """Two-rarefaction bound of Sec. 3.7 for unit vectors n (3, m)."""
    def project(U):
        rho = U[0]
        mt = (n * U[1:4]).sum(0)
        q = U[1:4] - mt * n
        Et = U[4] - (q * q).sum(0) / (2.0 * rho)
        u = mt / rho
        p = (GAMMA - 1.0) * (Et - mt * mt / (2.0 * rho))
        c = torch.sqrt(GAMMA * p / rho)
        return rho, u, p, c

    rL, uL, pL, cL = project(Ui)
    rR, uR, pR, cR = project(Uj)
    e = (GAMMA - 1.0) / (2.0 * GAMMA)
    num = cL + cR - 0.5 * (GAMMA - 1.0) * (uR - uL)
    num = torch.clamp(num, min=0.0)
    den = cL * (pL / pR) ** (-e) + cR
    p_tr = pR * (num / den) ** (1.0 / e)
    p_max = torch.maximum(pL, pR)

    def f(rho, p_side, c_side, p):
        shock = p >= p_side
        a = np.sqrt(2.0) * (p - p_side) / torch.sqrt(rho * ((GAMMA + 1.0) * p + (GAMMA - 1.0) * p_side))
        ratio = _safe(p / p_side, ~shock)
        b = (ratio ** ((GAMMA - 1.0) / (2.0 * GAMMA)) - 1.0) * 2.0 * c_side / (GAMMA - 1.0)
        return _where(shock, a, b)

    psi = f(rL, pL, cL, p_max) + f(rR, pR, cR, p_max) + uR - uL
    p_star = _where(psi < 0.0, p_tr, torch.minimum(p_max, p_tr))
    k = (GAMMA + 1.0) / (2.0 * GAMMA)
    lam1 = uL - cL * torch.sqrt(1.0 + k * torch.clamp((p_star - pL) / pL, min=0.0))
    lam3 = uR + cR * torch.sqrt(1.0 + k * torch.clamp((p_star - pR) / pR, min=0.0))
    return torch.maximum(torch.clamp(-lam1, min=0.0), torch.clamp(lam3, min=0.0))


def _rho_eps(V):
    return V[0] * V[4] - 0.5 * (V[1] ** 2 + V[2] ** 2 + V[3] ** 2)


def _psi(V, phi_min):
    return _rho_eps(V) - phi_min * _safe(V[0], V[0] > 0) ** (GAMMA + 1.0)


def _admissible(V, phi_min):
    scale = torch.abs(_rho_eps(V)) + torch.abs(phi_min * _safe(V[0], V[0] > 0) ** (GAMMA + 1.0))
    return _psi(V, phi_min) >= -1e-13 * scale


def _dpsi(V, P, phi_min):
    drho_eps = P[0] * V[4] + V[0] * P[4] - (V[1] * P[1] + V[2] * P[2] + V[3] * P[3])
    return drho_eps - phi_min * (GAMMA + 1.0) * _safe(V[0], V[0] > 0) ** GAMMA * P[0]


def limiter(U, P, rho_min, rho_max, phi_min, newton_max=2, newton_tol=1e-10, eps=np.finfo(np.float64).eps):
    """Alg. 2/3 over many entries at once (columns of U, P)."""
    rhoU, rhoP = U[0], P[0]
    nz = rhoP != 0.0
    absP = _safe(torch.abs(rhoP), nz)
    tR = torch.ones_like(rhoU)
    c1 = (rhoU + tR * rhoP > rho_max) & nz
    tR = _where(c1, torch.abs(rho_max - rhoU) / absP, tR)
    c2 = (rhoU + tR * rhoP < rho_min) & nz
    tR = _where(c2, torch.abs(rho_min - rhoU) / absP, tR)
    tR = torch.clamp(tR, 0.0, 1.0)
    tL = torch.zeros_like(rhoU)
    tol = newton_tol * _rho_eps(U)
    done = torch.zeros_like(rhoU, dtype=torch.bool)
    for _ in range(newton_max):
        VR = U + tR * P
        accept = ~done & _admissible(VR, phi_min)
        tL = _where(accept, tR, tL)
        done = done | accept
        VL = U + tL * P
        psiL = _psi(VL, phi_min)
        done = done | (psiL <= tol)
        act = ~done
        psiR = _psi(VR, phi_min)
        dL = _dpsi(VL, P, phi_min)
        dR = _dpsi(VR, P, phi_min)
        scaling = 1.0 / (tR - tL + eps)
        d12 = (psiR - psiL) * scaling
        d112 = (d12 - dL) * scaling
        d122 = (dR - d12) * scaling
        lamL = torch.clamp(dL * dL - 4.0 * psiL * d112, min=0.0)
        lamR = torch.clamp(dR * dR - 4.0 * psiR * d122, min=0.0)
        sL = _where(lamL > 0, torch.sqrt(_safe(lamL, lamL > 0)), torch.zeros_like(lamL))
        sR = _where(lamR > 0, torch.sqrt(_safe(lamR, lamR > 0)), torch.zeros_like(lamR))
        denL = dL - sL
        denR = dR - sR
        nL = tL - 2.0 * psiL / _safe(denL, act & (denL != 0))
        nR = tR - 2.0 * psiR / _safe(denR, act & (denR != 0))
        nL = _where(act & (denL != 0), nL, tL)
        nR = _where(act & (denR != 0), nR, tR)
        nL = torch.minimum(torch.maximum(nL, tL), tR)
        keep = _admissible(U + nL * P, phi_min)
        nL = _where(keep, nL, tL)
        nR = torch.minimum(torch.maximum(nR, nL), tR)
        tL = _where(act, nL, tL)
        tR = _where(act, nR, tR)
    return tL


def euler_step(tm: TorchMesh, U, tau=None, cfl=0.5, passes=2, newton_max=2, newton_tol=1e-10):
    """One euler_step (Alg. 1) with boundary post-processing; returns
    (U_out, tau).  tau=None computes tau_n (first RK stage)."""
    rows, col, off = tm.rows, tm.col, tm.off
    Ui, Uj = U[:, rows], U[:, col]
    # Step 1: d_ij = max of both orientations (symmetric), alpha_i (Sec. 3.8)
    nc = torch.sqrt((tm.c ** 2).sum(0))
    ncT = torch.sqrt((tm.cT ** 2).sum(0))
    lij = lambda_max(tm.c / _safe(nc, nc > 0), Ui, Uj) * nc
    lji = lambda_max(tm.cT / _safe(ncT, ncT > 0), Uj, Ui) * ncT
    d_off = _where(off, torch.maximum(lij, lji), torch.zeros_like(lij))
    d_ii = -tm.row_sum(d_off)
    d = _where(tm.diag, d_ii[rows], d_off)
    rho_eps = U[0] * internal_energy(U)
    eta = rho_eps ** (1.0 / (GAMMA + 1.0))
    s = eta / U[0]
    pre = rho_eps ** (-GAMMA / (GAMMA + 1.0)) / (GAMMA + 1.0)
    etap = torch.stack([pre * U[4], -pre * U[1], -pre * U[2], -pre * U[3], pre * U[0]])
    a = tm.row_sum((s[col] - s[rows]) * (Uj[1:4] * tm.c).sum(0))
    fj = flux_dot(Uj, tm.c)
    fi = flux_dot(Ui, tm.c)
    b = tm.row_sum(fj - fi)
    num = a - (etap * b).sum(0) + s * b[0]
    shift = torch.zeros_like(etap)
    shift[0] = s
    D = torch.abs(a) + (torch.abs(etap - shift) * torch.abs(b)).sum(0)
    alpha = _where(D > 0, torch.abs(num) / _safe(D, D > 0), torch.zeros_like(D))
    # Step 2: tau
    tau_max = torch.min(tm.mi / (-2.0 * d_ii))
    if tau is None:
        tau = cfl * tau_max
    # Step 3: low-order update, R, bounds
    dH = d * (alpha[rows] + alpha[col]) / 2.0
    R = tm.row_sum(-fj + dH * (Uj - Ui))
    nzd = d != 0
    ubar = 0.5 * (Ui + Uj) - (fj - fi) / (2.0 * _safe(d, nzd))
    coef = 2.0 * tau / tm.mi[rows] * d
    UL = U + tm.row_sum(_where(nzd, coef * ubar, torch.zeros_like(ubar)))
    big = torch.full_like(d, float("inf"))
    rho_min = torch.full((tm.n,), float("inf"), dtype=U.dtype).scatter_reduce(
        0, rows, _where(nzd, ubar[0], big), "amin", include_self=True)
    rho_max = torch.full((tm.n,), -float("inf"), dtype=U.dtype).scatter_reduce(
        0, rows, _where(nzd, ubar[0], -big), "amax", include_self=True)
    phi_min = torch.full((tm.n,), float("inf"), dtype=U.dtype).scatter_reduce(
        0, rows, specific_entropy(Uj), "amin", include_self=True)
    # Step 4: P_ij and limiter values
    lam = tm.lam
    b_ij = -tm.mij / tm.mi[col]
    b_ji = -tm.mij[tm.kT] / tm.mi[rows]
    P = tau / (tm.mi[rows] * lam[rows]) * (b_ij * R[:, col] - b_ji * R[:, rows] + (dH - d) * (Uj - Ui))
    P = _where(off, P, torch.zeros_like(P))
    bnd = (rho_min[rows], rho_max[rows], phi_min[rows])
    lim = limiter(UL[:, rows], P, *bnd, newton_max=newton_max, newton_tol=newton_tol)
    l = _where(off, lim, torch.zeros_like(lim))
    Ucur = UL
    for pss in range(1, passes + 1):
        lk = torch.minimum(l, l[tm.kT])
        Unext = Ucur + tm.row_sum(_where(off, lam[rows] * lk * P, torch.zeros_like(P)))
        if pss < passes:
            P = (1.0 - lk) * P
            lim = limiter(Unext[:, rows], P, *bnd, newton_max=newton_max, newton_tol=newton_tol)
            l = _where(off, lim, torch.zeros_like(lim))
        Ucur = Unext
    # boundary post-processing (Reading A20)
    out = Ucur
    if bool((tm.bc != 0).any()):
        comps = []
        inflow = (tm.bc & 8) != 0
        for f in range(NF):
            v = out[f]
            if 1 <= f <= 3:
                v = _where((tm.bc & (1 << (f - 1))) != 0, torch.zeros_like(v), v)
            v = _where(inflow, tm.inflow[f].expand_as(v), v)
            comps.append(v)
        out = torch.stack(comps)
    return out, tau


def ssprk3_step(tm, U, **kw):
    """SSP-RK3 (Sec. 3.6 eq. ssprk3) with tau fixed by the first stage."""
    U1, tau = euler_step(tm, U, **kw)
    E, _ = euler_step(tm, U1, tau=tau, **kw)
    U2 = 0.75 * U + 0.25 * E
    E, _ = euler_step(tm, U2, tau=tau, **kw)
    return 1.0 / 3.0 * U + 2.0 / 3.0 * E, tau
