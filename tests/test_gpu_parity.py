"""Parity of the CUDA stage (through the C ABI) with the FP64 oracle.

Tolerances: per field, 1e-12 relative in the 2-norm for one euler_step and
one SSP-RK3 step, and 1e-12 in the max-norm as well except on the isentropic
vortex (1e-11 there, see gpu_common.ISENTROPIC_MAX_TOL); 1e-9 in the max-norm
after 100 SSP-RK3 steps on smooth data; intermediate fields within
1e-13..1e-12 on the state scale.  The GPU
evaluates the same formulas in a different rounding order (FMA contraction,
reciprocal multiplies, Newton-refined powers), so bitwise equality is not
expected; the invariant checks hold exactly.
"""
import numpy as np
import pytest

import oracle as O
from gpu_common import ISENTROPIC_MAX_TOL, rel_field_err, rel_field_err_l2, require_gpu
from helpers import csr_rows, internal_energy, specific_entropy
from paper_2007_00094_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _mesh(name):
    if name == "vortex17":
        m = W.vortex_mesh(17)
        return m, W.vortex_state(m)
    if name == "wallbox_jitter":
        m = W.box_mesh((13, 11, 9), hi=(1.2, 1.0, 0.8), periodic=(False, False, False), jitter=0.25, seed=3)
        rho, u, p = W.vortex_primitive(m.x)
        U = W.primitive_to_conserved(rho, u, p)
        U[1:4] = np.where((m.bc & np.array([[1], [2], [4]])) > 0, 0.0, U[1:4])
        return m, U
    if name == "sod_jitter":
        m = W.box_mesh((40, 6, 5), periodic=(False, True, True), jitter=0.2, seed=5)
        return m, W.sod_state(m)
    if name == "ffs10":
        m = W.forward_step_mesh(m=10, jitter=0.2, seed=2007)
        U = W.forward_step_state(m)
        return m, U
    if name == "tiny3":
        m = W.vortex_mesh(3)
        return m, W.vortex_state(m)
    # 2D Q1 (quadrilaterals, 9-point stencil)
    if name == "bumpy2d_jitter":
        # density bumps make the entropy non-constant (see gpu_common on the isentropic case)
        m = W.rect_mesh((37, 29), periodic=(True, True), jitter=0.25, seed=8)
        return m, W.bumpy_vortex_state(m, amplitude=5e-2)
    if name == "wallrect_jitter":
        m = W.rect_mesh((41, 35), hi=(1.2, 1.0), periodic=(False, False), jitter=0.25, seed=9)
        U = W.riemann_state(m.x, (1.0, (0.3, -0.2, 0.0), 1.0), (0.2, (-0.5, 0.4, 0.0), 0.15),
                            normal=(0.8, 0.6, 0.0), point=(0.55, 0.45, 0.0))
        U[1:3] = np.where((m.bc & np.array([[1], [2]])) > 0, 0.0, U[1:3])
        return m, U
    if name == "ffs2d_10":
        m = W.forward_step_mesh_2d(m=10, jitter=0.2, seed=2007)
        return m, W.forward_step_state(m)
    raise KeyError(name)


CASES = ["vortex17", "wallbox_jitter", "sod_jitter", "ffs10", "tiny3", "bumpy2d_jitter", "wallrect_jitter",
         "ffs2d_10"]


def _isentropic(name):
    return name.startswith("vortex")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _solver(mesh, **kw):
    from paper_2007_00094_gb300.idp import Solver
    return Solver(mesh, **kw)


@pytest.mark.parametrize("name", CASES)
def test_matrices_match_oracle(name):
    mesh, _ = _mesh(name)
    s = _solver(mesh)
    om = O.assemble(mesh)
    rowptr, col, mij, cij, mi = s.matrices()
    np.testing.assert_array_equal(rowptr, om.rowptr)
    np.testing.assert_array_equal(col, om.col)
    assert np.abs(mij - om.mij).max() <= 1e-14 * np.abs(om.mij).max()
    assert np.abs(cij - om.cij).max() <= 1e-14 * np.abs(om.cij).max()
    assert np.abs(mi - om.mi).max() <= 1e-14 * np.abs(om.mi).max()


@pytest.mark.parametrize("name", CASES)
def test_euler_step_trace_parity(name, n_threads):
    mesh, U = _mesh(name)
    om = O.assemble(mesh)
    ref, tau_ref, st, tr = O.euler_step(om, U, params=O.default_params(n_threads=n_threads), trace=True)
    assert st == 0
    s = _solver(mesh)
    s.init_state(U)
    tau = s.euler_step(trace=True)
    assert abs(tau - tau_ref) <= 1e-14 * tau_ref
    assert abs(s.field("tau_max") - tr["tau_max"]) <= 1e-14 * tr["tau_max"]
    d = s.field("d")
    assert np.abs(d - tr["d"]).max() <= 1e-13 * np.abs(tr["d"]).max()
    rows = csr_rows(om)
    off = rows != om.col
    Umax = np.abs(U).max()
    # alpha is a ratio of round-off sized numbers where the state is nearly
    # constant; it matters through d^H_ij (U_j - U_i), so its error is
    # weighted by the local variation of U
    var = np.zeros(om.n)
    np.maximum.at(var, rows, np.abs(U[:, om.col] - U[:, rows]).max(axis=0) / Umax)
    assert (np.abs(s.field("alpha") - tr["alpha"]) * var).max() <= 1e-12
    # state-sized quantities against the state scale
    max_tol = ISENTROPIC_MAX_TOL if _isentropic(name) else 1e-12
    for key, tol in (("UL", 1e-13), ("bounds", 1e-13), ("U5", max_tol), ("Ulim", max_tol)):
        err = rel_field_err(s.field(key), tr[key])
        assert err.max() <= tol, (key, err)
    for key in ("U5", "Ulim"):
        assert rel_field_err_l2(s.field(key), tr[key]).max() <= 1e-12, key
    # R enters the update as tau R_i / m_i, P_ij as lambda l_ij P_ij: both are
    # state increments and are compared on the state scale
    dR = np.abs(s.field("R") - tr["R"]) * (tau_ref / om.mi)[None, :]
    assert dR.max() <= 1e-13 * Umax
    P = s.field("P")
    assert np.abs(P - tr["P"]).max() <= 1e-13 * Umax
    # limiter values: where the limiter's decision is a tie at rounding level
    # (P itself at rounding level, or Psi within its rounding error) both
    # values are admissible; compare l_ij weighted by the size of P_ij
    Pn = np.abs(P).max(axis=0) / Umax
    for key in ("l4", "l5"):
        dl = np.abs(s.field(key) - tr[key])[off]
        assert (dl * Pn[off]).max() <= (1e-9 if _isentropic(name) else 1e-11), key
    out = s.get_state()
    assert rel_field_err(out, ref).max() <= max_tol
    assert rel_field_err_l2(out, ref).max() <= 1e-12


@pytest.mark.parametrize("name", CASES)
def test_rk3_step_parity_and_invariants(name, n_threads):
    mesh, U = _mesh(name)
    om = O.assemble(mesh)
    prm = O.default_params(n_threads=n_threads)
    s = _solver(mesh)
    s.init_state(U)
    ref = U
    for _ in range(3):
        ref, tau, st = O.ssprk3_step(om, ref, prm)
        assert st == 0
    s.step(3)
    s.synchronize()
    out = s.get_state()
    assert rel_field_err(out, ref).max() <= (ISENTROPIC_MAX_TOL if _isentropic(name) else 1e-12)
    assert rel_field_err_l2(out, ref).max() <= 1e-12
    assert (out[0] > 0).all() and (internal_energy(out) > 0).all()
    st, rep = s.check_bounds()
    assert st == 0 and rep.n_rho_nonpositive == 0 and rep.n_eps_nonpositive == 0
    if mesh.dim == 2:  # c_ij has no z component: m_z = 0 stays exactly 0
        assert not out[3].any()


def test_local_bounds_hold_on_gpu():
    mesh, U = _mesh("sod_jitter")
    s = _solver(mesh)
    s.init_state(U)
    for _ in range(5):
        s.euler_step(trace=True)
        ulim, bnd = s.field("Ulim"), s.field("bounds")
        slack = 1e-12
        assert (ulim[0] >= bnd[0] - slack * np.abs(bnd[0])).all()
        assert (ulim[0] <= bnd[1] + slack * np.abs(bnd[1])).all()
        assert (specific_entropy(ulim) >= bnd[2] - slack * np.abs(bnd[2])).all()


def test_hundred_steps_smooth_vortex(n_threads):
    mesh = W.vortex_mesh(17)
    U = W.vortex_state(mesh)
    om = O.assemble(mesh)
    ref, t_ref, _ = O.run(om, U, 100, O.default_params(n_threads=n_threads))
    s = _solver(mesh)
    s.init_state(U)
    s.step(100)
    s.synchronize()
    out = s.get_state()
    t, _ = s.time()
    assert abs(t - t_ref) <= 1e-12 * t_ref
    err = rel_field_err(out, ref)
    assert err.max() <= 1e-9, err


def test_conservation_on_gpu():
    mesh = W.box_mesh((12, 11, 5), periodic=(True, True, True), jitter=0.2, seed=7)
    U = W.vortex_state(mesh)
    s = _solver(mesh)
    s.init_state(U)
    mi = s.matrices()[4]
    before = (mi[None] * U).sum(axis=1)
    s.step(10)
    s.synchronize()
    after = (mi[None] * s.get_state()).sum(axis=1)
    scale = (mi[None] * np.abs(U)).sum(axis=1).max()
    assert np.abs(after - before).max() <= 1e-12 * scale


def test_deterministic():
    mesh, U = _mesh("ffs10")
    outs = []
    for _ in range(2):
        s = _solver(mesh)
        s.init_state(U)
        s.step(5)
        s.synchronize()
        outs.append(s.get_state())
    np.testing.assert_array_equal(outs[0], outs[1])


def test_mesh_upload_rejects_invalid_meshes():
    """Empty meshes, node ids out of range, a node in no cell and an inverted
    cell are reported (IDP_ERR_ARG) at upload, for hexahedra and quadrilaterals."""
    import copy
    from paper_2007_00094_gb300.idp import IdpError
    for base in (W.box_mesh((4, 3, 3), periodic=(False, False, False)), W.rect_mesh((4, 3), periodic=(False, False))):
        bad = []
        m = copy.deepcopy(base)
        m.cells = m.cells[:0]
        m.cell_xyz = m.cell_xyz[:0]
        bad.append(m)
        m = copy.deepcopy(base)
        m.cells[0, 0] = m.n_nodes  # out of range
        bad.append(m)
        m = copy.deepcopy(base)
        m.x = np.vstack([m.x, m.x[:1]])  # one more node that no cell uses
        m.bc = np.append(m.bc, 0).astype(np.int32)
        bad.append(m)
        m = copy.deepcopy(base)
        m.cell_xyz[0, :, 0] = -m.cell_xyz[0, :, 0]  # mirrored in x: negative Jacobian
        bad.append(m)
        for m in bad:
            with pytest.raises(IdpError) as e:
                _solver(m)
            assert e.value.status == 1  # IDP_ERR_ARG


def test_rejects_inadmissible_state():
    from paper_2007_00094_gb300.idp import IdpError
    mesh, U = _mesh("tiny3")
    s = _solver(mesh)
    bad = U.copy()
    bad[0, 5] = -1.0
    with pytest.raises(IdpError) as e:
        s.init_state(bad)
    assert e.value.status == 4
    bad = U.copy()
    bad[4, 7] = 0.0  # epsilon < 0
    with pytest.raises(IdpError):
        s.init_state(bad)


def test_cfl_violation_reported():
    from paper_2007_00094_gb300.idp import IdpError
    mesh, U = _mesh("vortex17")
    s = _solver(mesh)
    s.init_state(U)
    s.euler_step(trace=True)
    tmax = s.field("tau_max")
    s.init_state(U)
    with pytest.raises(IdpError) as e:
        s.euler_step(tau=tmax * 1.5)
    assert e.value.status == 5


def test_torch_device_buffers():
    import torch
    mesh, U = _mesh("vortex17")
    s = _solver(mesh)
    Ud = torch.from_numpy(U).cuda().contiguous()
    s.init_state(Ud)
    s.step(2)
    out = torch.empty_like(Ud)
    s.get_state(out)
    torch.cuda.synchronize()
    s2 = _solver(mesh)
    s2.init_state(U)
    s2.step(2)
    np.testing.assert_array_equal(out.cpu().numpy(), s2.get_state())


@pytest.mark.parametrize("name", ["wallbox_jitter", "sod_jitter", "vortex17", "wallrect_jitter"])
def test_relaxed_bounds_parity(name, n_threads):
    """Bound relaxation (idp_config.relax, Reading A14) against the oracle with
    the same option: the relaxed bounds, one euler_step and one SSP-RK3 step."""
    mesh, U = _mesh(name)
    om = O.assemble(mesh)
    prm = O.default_params(n_threads=n_threads, relax=1)
    ref, tau_ref, st, tr = O.euler_step(om, U, params=prm, trace=True)
    assert st == 0
    s = _solver(mesh, relax=1)
    s.init_state(U)
    tau = s.euler_step(trace=True)
    assert abs(tau - tau_ref) <= 1e-14 * tau_ref
    b = s.field("bounds")
    assert np.abs(b - tr["bounds"]).max() <= 1e-13 * np.abs(tr["bounds"]).max()
    out = s.get_state()
    assert rel_field_err_l2(out, ref).max() <= 1e-12
    ref3, _, st = O.ssprk3_step(om, U, prm)
    s.init_state(U)
    s.step(1)
    s.synchronize()
    assert rel_field_err_l2(s.get_state(), ref3).max() <= 1e-12
