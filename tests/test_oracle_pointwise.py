"""Pins for the oracle's pointwise building blocks.

* lambda~_max (Sec. 3.7): equal-state closed form |u| + c, the orientation
  symmetry, and brute force against an exact Riemann solver (bisection for
  p*): the bound never falls below the exact maximum wavespeed and is exact
  when both waves are rarefactions.
* Harten entropy derivative (Sec. 3.8, Reading A7) by central differences.
* Limiter (Alg. 2/3): the returned t keeps U + tP inside the local bounds,
  t = 1 whenever U + P is admissible, and t never exceeds the largest
  admissible t found by bisection.
"""
import math

import numpy as np
import pytest

import oracle as O
from exact_riemann import max_wave_speed
from helpers import rho_eps, specific_entropy
from paper_2007_00094_gb300.workloads import primitive_to_conserved


def _state(rho, u, p):
    return primitive_to_conserved(np.array([rho]), np.array(u, float).reshape(3, 1), np.array([p]))[:, 0]


def test_lambda_max_equal_states():
    rng = np.random.default_rng(1)
    for _ in range(200):
        rho, p = rng.uniform(0.05, 5.0), rng.uniform(0.05, 10.0)
        u = rng.uniform(-4, 4, size=3)
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        U = _state(rho, u, p)
        lam = O.lambda_max(n, U, U)
        expect = abs(u @ n) + math.sqrt(1.4 * p / rho)
        assert abs(lam - expect) <= 1e-14 * expect


def test_lambda_max_orientation_symmetry():
    rng = np.random.default_rng(2)
    for _ in range(300):
        Ui = _state(rng.uniform(0.1, 2), rng.uniform(-2, 2, 3), rng.uniform(0.1, 10))
        Uj = _state(rng.uniform(0.1, 2), rng.uniform(-2, 2, 3), rng.uniform(0.1, 10))
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        a = O.lambda_max(n, Ui, Uj)
        b = O.lambda_max(-n, Uj, Ui)
        assert abs(a - b) <= 1e-13 * a


def test_lambda_max_brute_force_upper_bound():
    """Grid of 1D states: rho, p log-spaced in [1e-2, 1e2], u in [-5, 5]."""
    rhos = np.geomspace(1e-2, 1e2, 5)
    ps = np.geomspace(1e-2, 1e2, 5)
    us = np.linspace(-5, 5, 5)
    n = np.array([1.0, 0.0, 0.0])
    worst = np.inf
    n_rare = 0
    for rL in rhos:
        for pL in ps:
            for uL in us:
                UL = _state(rL, (uL, 0.3, -0.2), pL)
                for rR in rhos:
                    for pR in ps:
                        for uR in us:
                            UR = _state(rR, (uR, -0.1, 0.5), pR)
                            lam = O.lambda_max(n, UL, UR)
                            exact, pstar = max_wave_speed((rL, uL, pL), (rR, uR, pR))
                            worst = min(worst, (lam - exact) / exact)
                            assert lam >= exact * (1.0 - 1e-12), (rL, uL, pL, rR, uR, pR)
                            if 0 < pstar < min(pL, pR) * (1 - 1e-9):
                                n_rare += 1  # two rarefactions: the bound is exact
                                assert abs(lam - exact) <= 1e-9 * exact
    assert n_rare > 100
    assert worst > -1e-12


def test_entropy_derivative_finite_differences():
    rng = np.random.default_rng(3)
    for _ in range(20):
        U = _state(rng.uniform(0.2, 3), rng.uniform(-2, 2, 3), rng.uniform(0.2, 5))
        q = O.node_quantities(U)
        etap = q[4:9]
        for k in range(5):
            h = 1e-6 * max(1.0, abs(U[k]))
            Up, Um = U.copy(), U.copy()
            Up[k] += h
            Um[k] -= h
            fd = (O.node_quantities(Up)[3] - O.node_quantities(Um)[3]) / (2 * h)
            assert abs(fd - etap[k]) <= 1e-7 * (abs(etap).max())
        # eta = (rho eps)^(1/(gamma+1)), phi = eps rho^-gamma, p = 0.4 eps
        eps = U[4] - 0.5 * (U[1:4] ** 2).sum() / U[0]
        assert abs(q[0] - 0.4 * eps) < 1e-14 * q[0]
        assert abs(q[3] - (U[0] * eps) ** (1 / 2.4)) < 1e-14 * q[3]
        assert abs(q[2] - eps / U[0] ** 1.4) < 1e-14 * q[2]


def test_psi_definition():
    rng = np.random.default_rng(4)
    for _ in range(50):
        U = _state(rng.uniform(0.2, 3), rng.uniform(-2, 2, 3), rng.uniform(0.2, 5))
        phi_min = rng.uniform(0.1, 2.0)
        literal = U[0] ** 2.4 * (specific_entropy(U) - phi_min)
        assert abs(O.psi(U, phi_min) - literal) <= 1e-13 * abs(rho_eps(U))


def _admissible(V, rmin, rmax, pmin, slack=1e-12):
    r = V[0]
    ok_r = (r >= rmin - slack * abs(rmin)) and (r <= rmax + slack * abs(rmax))
    return ok_r and rho_eps(V) - pmin * r ** 2.4 >= -slack * abs(rho_eps(V))


def _bisect_tstar(U, P, rmin, rmax, pmin):
    if _admissible(U + P, rmin, rmax, pmin, 0.0):
        return 1.0
    lo, hi = 0.0, 1.0
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        if _admissible(U + mid * P, rmin, rmax, pmin, 0.0):
            lo = mid
        else:
            hi = mid
    return hi


@pytest.mark.parametrize("newton_max", [2, 8])
def test_limiter_admissible_and_below_bisection(newton_max):
    rng = np.random.default_rng(5 + newton_max)
    prm = O.default_params(newton_max=newton_max)
    n_limited = 0
    for trial in range(3000):
        U = _state(rng.uniform(0.2, 3), rng.uniform(-2, 2, 3), rng.uniform(0.2, 5))
        r = U[0]
        rmin = r * rng.uniform(0.6, 1.0)
        rmax = r * rng.uniform(1.0, 1.5)
        phi = specific_entropy(U)
        pmin = phi * rng.uniform(0.5, 1.0)
        P = rng.normal(size=5) * U * rng.choice([0.01, 0.1, 0.5, 2.0])
        t = O.limiter(U, P, rmin, rmax, pmin, prm)
        assert 0.0 <= t <= 1.0
        V = U + t * P
        assert _admissible(V, rmin, rmax, pmin, 1e-12), (trial, t)
        tstar = _bisect_tstar(U, P, rmin, rmax, pmin)
        assert t <= tstar + 1e-12
        if _admissible(U + P, rmin, rmax, pmin, 0.0):
            assert t == 1.0
        else:
            n_limited += 1
    assert n_limited > 500


def test_limiter_newton_converges_with_more_steps():
    """For rho(P) > 0 the third derivative of Psi along U + tP is negative, so
    the quadratic Newton step of Alg. 3 keeps the root bracketed and converges
    to the bisection root as the step count grows.  (For rho(P) < 0 the step
    crosses the root and the safeguards return an admissible, smaller t.)"""
    rng = np.random.default_rng(11)
    gaps = {1: [], 2: [], 3: [], 8: []}
    for _ in range(400):
        U = _state(rng.uniform(0.5, 2), rng.uniform(-1, 1, 3), rng.uniform(0.5, 2))
        phi = specific_entropy(U)
        P = rng.normal(size=5) * U * 0.5
        P[0] = abs(P[0])
        tstar = _bisect_tstar(U, P, 0.0, 1e9, phi * 0.999)
        for k in gaps:
            t = O.limiter(U, P, 0.0, 1e9, phi * 0.999, O.default_params(newton_max=k, newton_tol=0.0))
            assert t <= tstar + 1e-12
            gaps[k].append(tstar - t)
    means = [np.mean(gaps[k]) for k in sorted(gaps)]
    assert all(a >= b for a, b in zip(means, means[1:]))
    assert np.max(gaps[2]) < 1e-2
    assert np.max(gaps[8]) < 1e-12


@pytest.mark.parametrize("newton_max", [1, 2])
def test_limiter_is_exact_where_psi_is_quadratic(newton_max):
    """With rho(P) = 0 the density is constant along U + tP, so
    Psi(t) = rho eps(U + tP) - phi_min rho^(gamma+1) is the quadratic
    c + b t + a t^2 with a = -|P_m|^2/2, b = rho P_E - m.P_m, c = Psi(0).
    Alg. 3's step solves the quadratic through the bracket's values, slopes and
    second divided differences, which is Psi itself here: at the default Newton
    settings the limiter must return the positive root
    t* = (b + sqrt(b^2 - 4ac)) / (-2a), from the quadratic formula, whenever
    Psi(0) > 0 > Psi(1).  (The Psi margin of Reading A27 moves t by far less
    than the tolerance.)"""
    rng = np.random.default_rng(23 + newton_max)
    prm = O.default_params(newton_max=newton_max)
    n = 0
    for _ in range(2000):
        U = _state(rng.uniform(0.2, 3), rng.uniform(-2, 2, 3), rng.uniform(0.2, 5))
        rho, m = U[0], U[1:4]
        pmin = specific_entropy(U) * rng.uniform(0.3, 0.999)
        P = rng.normal(size=5) * np.abs(U) * rng.choice([0.1, 0.5, 2.0])
        P[0] = 0.0
        a = -0.5 * float(P[1:4] @ P[1:4])
        b = rho * P[4] - float(m @ P[1:4])
        c = rho_eps(U) - pmin * rho ** 2.4
        if not (c > 0.0 and a + b + c < 0.0):
            continue  # the root must lie inside (0, 1)
        tstar = (b + np.sqrt(b * b - 4.0 * a * c)) / (-2.0 * a)
        t = O.limiter(U, P, 0.0, 1e9, pmin, prm)
        assert abs(t - tstar) <= 1e-9 * tstar, (t, tstar)
        n += 1
    assert n > 500
