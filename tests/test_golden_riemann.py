"""The test-side exact Riemann solver against published star-region values.

This pins the independent reference that the Sod convergence test of the
oracle relies on (tests/golden/sod_star_state.json, with its citation).
"""
import json
import os

from exact_riemann import sample, star_pressure

HERE = os.path.dirname(os.path.abspath(__file__))


def test_sod_star_region():
    with open(os.path.join(HERE, "golden", "sod_star_state.json")) as fh:
        g = json.load(fh)
    L = (g["left"]["rho"], g["left"]["u"], g["left"]["p"])
    R = (g["right"]["rho"], g["right"]["u"], g["right"]["p"])
    p, u = star_pressure(L, R, g["gamma"])
    tol = 0.5 * 10.0 ** (-g["digits"])
    assert abs(p - g["p_star"]) < tol
    assert abs(u - g["u_star"]) < tol
    # densities either side of the contact, sampled just left / right of u*
    rl = sample(L, R, [u - 1e-9], g["gamma"])[0, 0]
    rr = sample(L, R, [u + 1e-9], g["gamma"])[0, 0]
    assert abs(rl - g["rho_star_left"]) < tol
    assert abs(rr - g["rho_star_right"]) < tol
