"""Pins for the Psi margin of the oracle's limiter (Reading A27).

Alg. 2 accepts a line-search point when Psi >= 0.  The caption of Alg. 3
states that an implementation has to add safeguards against round-off; the
oracle takes Psi >= -1e-13 (|rho eps| + |phi_min rho^(gamma+1)|) as
admissible.  These tests show what that margin does and does not change, on
the limiter inputs (U^L_i or the pass-1 state, P_ij, the bounds of row i)
that the oracle's own euler_step produces:

- the margin changes a limiter value only where one of the limiter's
  admissibility tests saw a Psi inside [-margin, 0) of its scale; everywhere
  else margin 0 and margin 1e-13 agree bitwise;
- with the margin, rounding-level perturbations of the inputs (1e-15
  relative) no longer flip limiter decisions between accepting and rejecting,
  while the strict test flips hundreds (vortex) to thousands (Sod plateaus) of
  them;
- on the isentropic vortex, even with the margin, the limiter's root is so
  ill-conditioned that a 1e-15 relative perturbation of its inputs moves
  l_ij |P_ij| / |U| by more than 1e-11, which is why the parity tests weight
  limiter values by |P_ij| and take the stage's own sensitivity into account
  on that case.
"""
import numpy as np
import pytest

import oracle as O
from helpers import csr_rows, transpose_index
from paper_2007_00094_gb300 import workloads as W


def _wallbox():
    m = W.box_mesh((13, 11, 9), hi=(1.2, 1.0, 0.8), periodic=(False, False, False), jitter=0.25, seed=3)
    rho, u, p = W.vortex_primitive(m.x)
    U = W.primitive_to_conserved(rho, u, p)
    U[1:4] = np.where((m.bc & np.array([[1], [2], [4]])) > 0, 0.0, U[1:4])
    return m, U


def _case(name):
    if name == "vortex17":
        m = W.vortex_mesh(17)
        return m, W.vortex_state(m)
    if name == "sod_jitter":
        m = W.box_mesh((40, 6, 5), periodic=(False, True, True), jitter=0.2, seed=5)
        return m, W.sod_state(m)
    if name == "wallbox_jitter":
        return _wallbox()
    raise KeyError(name)


_CACHE = {}


def _limiter_inputs(name, n_threads):
    """(U, P, bounds, l, Pn, Umax) of every off-diagonal limiter call of Step 4
    and of limiter pass 1 of one oracle euler_step."""
    if name in _CACHE:
        return _CACHE[name]
    mesh, U = _case(name)
    om = O.assemble(mesh)
    _, _, st, tr = O.euler_step(om, U, params=O.default_params(n_threads=n_threads), trace=True)
    assert st == 0
    rows = csr_rows(om)
    off = rows != om.col
    kT = transpose_index(om)
    lmin = np.minimum(tr["l4"], tr["l4"][kT])
    out = {}
    for stage, Us, P in (("l4", tr["UL"], tr["P"]), ("l5", tr["U5"], (1.0 - lmin) * tr["P"])):
        out[stage] = (Us[:, rows[off]], P[:, off], tr["bounds"][:, rows[off]], tr[stage][off],
                      np.abs(P[:, off]).max(axis=0) / np.abs(U).max())
    _CACHE[name] = out
    return out


@pytest.mark.parametrize("name", ["vortex17", "sod_jitter", "wallbox_jitter"])
@pytest.mark.parametrize("stage", ["l4", "l5"])
def test_margin_changes_only_calls_it_decided(name, stage, n_threads):
    Ui, P, B, l_trace, _ = _limiter_inputs(name, n_threads)[stage]
    t_m, hits, worst = O.limiter_many(Ui, P, B, O.default_params())
    t_s, hits_s, _ = O.limiter_many(Ui, P, B, O.default_params(psi_margin=0.0))
    # the batched call reproduces the values of the stage itself
    np.testing.assert_array_equal(t_m, l_trace)
    differ = t_m != t_s
    # every difference comes from a test the margin decided ...
    assert not (differ & (hits == 0)).any()
    # ... and such a test saw |Psi| within the margin of its scale
    assert worst.max() <= 1e-13
    assert (hits_s == 0).all()  # the strict test never counts margin decisions
    # where the margin decided nothing, both give bitwise the same value
    np.testing.assert_array_equal(t_m[hits == 0], t_s[hits == 0])
    # the margin matters on these inputs (this is not a vacuous pin)
    assert differ.sum() >= 100


@pytest.mark.parametrize("name, strict_min", [("vortex17", 300), ("sod_jitter", 5000)])
def test_margin_makes_decisions_robust_to_rounding(name, strict_min, n_threads):
    """Perturb every limiter input by 1e-15 relative noise (a different but
    equally valid rounding of the stage): with the strict test hundreds to
    thousands of limiter values jump by more than 1e-3 (an acceptance turned
    into a rejection or back); with the margin none do."""
    rng = np.random.default_rng(2027)
    for stage in ("l4", "l5"):
        Ui, P, B, _, _ = _limiter_inputs(name, n_threads)[stage]
        Up = Ui * (1.0 + 1e-15 * rng.standard_normal(Ui.shape))
        Pp = P * (1.0 + 1e-15 * rng.standard_normal(P.shape))
        flips = {}
        for margin in (0.0, 1e-13):
            prm = O.default_params(psi_margin=margin)
            a, _, _ = O.limiter_many(Ui, P, B, prm)
            b, _, _ = O.limiter_many(Up, Pp, B, prm)
            flips[margin] = int((np.abs(a - b) > 1e-3).sum())
        assert flips[1e-13] == 0, (stage, flips)
        assert flips[0.0] >= strict_min, (stage, flips)


def test_isentropic_limiter_is_ill_conditioned(n_threads):
    """On the isentropic vortex phi is constant, so Psi(t) along U + tP is flat
    near its root: a 1e-15 relative input perturbation moves the returned t
    by far more than the input.  Weighted by |P_ij| / |U| the change exceeds
    1e-11 (the weighted limiter tolerance of the non-isentropic parity cases)
    but stays below 1e-9; on the Sod tube it stays below 1e-13."""
    rng = np.random.default_rng(7)
    moved = {}
    for name in ("vortex17", "sod_jitter"):
        m = 0.0
        for stage in ("l4", "l5"):
            Ui, P, B, _, Pn = _limiter_inputs(name, n_threads)[stage]
            Up = Ui * (1.0 + 1e-15 * rng.standard_normal(Ui.shape))
            Pp = P * (1.0 + 1e-15 * rng.standard_normal(P.shape))
            a, _, _ = O.limiter_many(Ui, P, B)
            b, _, _ = O.limiter_many(Up, Pp, B)
            m = max(m, float((np.abs(a - b) * Pn).max()))
        moved[name] = m
    assert 1e-11 < moved["vortex17"] < 1e-9, moved
    assert moved["sod_jitter"] < 1e-13, moved
