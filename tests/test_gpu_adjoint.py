"""The CUDA discrete adjoint (through the C ABI) against the reference
gradient: torch.autograd through the differentiable FP64 restatement of the
stage (oracle/torch_stage.py), on the same seeded inputs; and against central
differences of the CUDA forward run.

Both sides differentiate the same piecewise smooth map and take the branch
of their own forward pass at every kink, so they agree to rounding except
where rounding moves a forward value across a kink.  At an exact tie (two
equal candidates of a min or max, e.g. bitwise equal neighbour states of
z-invariant data) the derivative is not unique: torch splits it evenly
between the candidates, the CUDA adjoint gives it to one of them; both are
generalised gradients.  The inputs below are jittered meshes with seeded
non-symmetric data, where exact ties do not occur.
Tolerance: per field, 1e-11 relative in the 2-norm against the reference
gradient.  Measured on a GB300: at most 2e-13 (2-norm) and 5e-13 (max-norm)
for one stage and for three SSP-RK3 steps; the margin covers the limiter's
Newton derivatives, which amplify rounding of the traced values by
1/Psi'(t).
"""
import numpy as np
import pytest

from gpu_common import rel_field_err_l2, require_gpu
from paper_2007_00094_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ADJ_TOL = 1e-11


def _perturb(mesh, U, amp, seed):
    """Seeded perturbation of density, velocity and pressure.  The indicator
    alpha_i = N_i/D_i has derivatives of order 1/D_i; on an exactly constant
    state D_i is made of rounding noise, and so is the gradient, on either
    side.  Perturbed data keep D_i well above rounding."""
    rng = np.random.default_rng(seed)
    n = mesh.n_nodes
    rho = U[0] * (1.0 + amp * rng.standard_normal(n))
    u = U[1:4] / U[0] + amp * rng.standard_normal((3, n))
    eps = U[4] - 0.5 * (U[1] ** 2 + U[2] ** 2 + U[3] ** 2) / U[0]
    p = 0.4 * eps * (1.0 + amp * rng.standard_normal(n))
    u = np.where((mesh.bc & np.array([[1], [2], [4]])) > 0, 0.0, u)
    if mesh.dim == 2:
        u[2] = 0.0
    return W.primitive_to_conserved(rho, u, p)


def _case(name):
    if name == "vortex":
        m = W.vortex_mesh(7, nz=4, jitter=0.2, seed=11)
        return m, W.bumpy_vortex_state(m)
    if name == "wallbox":
        # the vortex is z-invariant: z-neighbours would hold bitwise equal
        # states, where bounds and wavespeeds tie exactly (see the module
        # docstring); the perturbation removes the ties
        m = W.box_mesh((6, 5, 5), periodic=(False, False, False), jitter=0.2, seed=3)
        rho, u, p = W.vortex_primitive(m.x)
        return m, _perturb(m, W.primitive_to_conserved(rho, u, p), 1e-3, 10)
    if name == "sod":
        m = W.box_mesh((14, 3, 3), periodic=(False, True, True), jitter=0.15, seed=5)
        return m, _perturb(m, W.sod_state(m), 1e-2, 8)
    if name == "ffs":
        m = W.forward_step_mesh(m=10, jitter=0.2, seed=2007)
        return m, _perturb(m, W.forward_step_state(m), 1e-2, 9)
    if name == "rect2d":
        m = W.rect_mesh((9, 8), hi=(1.1, 0.9), periodic=(False, False), jitter=0.2, seed=12)
        rho, u, p = W.vortex_primitive(m.x)
        return m, _perturb(m, W.primitive_to_conserved(rho, u, p), 1e-3, 13)
    if name == "ffs2d":
        m = W.forward_step_mesh_2d(m=10, jitter=0.2, seed=2007)
        return m, _perturb(m, W.forward_step_state(m), 1e-2, 14)
    raise KeyError(name)


CASES = ["vortex", "wallbox", "sod", "ffs", "rect2d", "ffs2d"]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _solver(mesh, **kw):
    from paper_2007_00094_gb300.idp import Solver
    return Solver(mesh, **kw)


def _torch_mesh(mesh):
    import oracle as O
    from oracle import torch_stage as T
    return T, T.TorchMesh(O.assemble(mesh))


def _weights(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


@pytest.mark.parametrize("fixed_tau", [False, True])
@pytest.mark.parametrize("name", CASES)
def test_adjoint_euler_step_matches_reference_gradient(name, fixed_tau):
    mesh, U = _case(name)
    T, tm = _torch_mesh(mesh)
    w = _weights(U.shape, 1)
    Ut = torch.as_tensor(U).clone().requires_grad_(True)
    if fixed_tau:
        _, tau0 = T.euler_step(tm, torch.as_tensor(U))
        tau_t = (0.8 * tau0).detach().clone().requires_grad_(True)
        out, _ = T.euler_step(tm, Ut, tau=tau_t)
        gU_ref, gtau_ref = torch.autograd.grad((torch.as_tensor(w) * out).sum(), (Ut, tau_t))
        tau = float(tau_t.detach())
    else:
        out, _ = T.euler_step(tm, Ut)
        (gU_ref,) = torch.autograd.grad((torch.as_tensor(w) * out).sum(), (Ut,))
        tau = None
    s = _solver(mesh)
    gU, gtau = s.adjoint_euler_step(U, w, tau=tau)
    err = rel_field_err_l2(gU, gU_ref.numpy())
    assert np.all(np.isfinite(gU))
    assert err.max() <= ADJ_TOL, err
    if fixed_tau:
        assert abs(gtau - float(gtau_ref)) <= ADJ_TOL * max(abs(float(gtau_ref)), 1e-300), (gtau, float(gtau_ref))


@pytest.mark.parametrize("name", ["wallbox", "sod", "vortex", "rect2d"])
def test_adjoint_rk3_run_matches_reference_gradient(name):
    """Three SSP-RK3 steps, checkpoints every second step (two segments)."""
    mesh, U = _case(name)
    T, tm = _torch_mesh(mesh)
    w = _weights(U.shape, 2)
    U0 = torch.as_tensor(U).clone().requires_grad_(True)
    V = U0
    for _ in range(3):
        V, _ = T.ssprk3_step(tm, V)
    (g_ref,) = torch.autograd.grad((torch.as_tensor(w) * V).sum(), (U0,))
    s = _solver(mesh)
    s.init_state(U)
    s.adjoint_record(3, checkpoint_every=2)
    # the recorded forward run is the ordinary one
    assert np.abs(s.get_state() - V.detach().numpy()).max() <= 1e-11 * np.abs(U).max()
    g = s.adjoint_backward(w)
    err = rel_field_err_l2(g, g_ref.numpy())
    assert err.max() <= ADJ_TOL, err


def test_adjoint_checkpoint_spacing_does_not_change_result():
    mesh, U = _case("sod")
    w = _weights(U.shape, 3)
    out = []
    for every in (1, 2, 4):
        s = _solver(mesh)
        s.init_state(U)
        s.adjoint_record(4, checkpoint_every=every)
        out.append(s.adjoint_backward(w))
    np.testing.assert_array_equal(out[0], out[1])
    np.testing.assert_array_equal(out[0], out[2])


@pytest.mark.parametrize("name", ["sod", "ffs2d"])
def test_stored_stage_traces_give_the_recomputed_gradient(name):
    """idp_config.adjoint_store_stages: the backward sweep over traces stored
    during the segment recompute equals, bitwise, the sweep that re-traces
    each stage before its reverse (both with checkpoint segments of 3 and a
    ragged last segment)."""
    mesh, U = _case(name)
    w = _weights(U.shape, 4)
    out = []
    for store in (1, 0):
        s = _solver(mesh, adjoint_store_stages=store)
        s.init_state(U)
        s.adjoint_record(5, checkpoint_every=3)
        out.append(s.adjoint_backward(w))
    np.testing.assert_array_equal(out[0], out[1])
    assert np.all(np.isfinite(out[0])) and np.abs(out[0]).max() > 0.0


def test_adjoint_is_deterministic_and_keeps_state():
    mesh, U = _case("wallbox")
    w = _weights(U.shape, 4)
    s = _solver(mesh)
    s.init_state(U)
    s.adjoint_record(2, checkpoint_every=1)
    U_end = s.get_state().copy()
    t_end = s.time()
    g1 = s.adjoint_backward(w)
    g2 = s.adjoint_backward(w)
    np.testing.assert_array_equal(g1, g2)
    np.testing.assert_array_equal(s.get_state(), U_end)
    assert s.time() == t_end


def test_adjoint_directional_derivative_matches_central_differences():
    """<g, v> against (J(U + eps v) - J(U - eps v)) / (2 eps) of the CUDA
    forward run.  The map is piecewise smooth; as for the reference gradient,
    a difference of width 2e-6 relative can straddle some branch points, so
    agreement is checked to 1e-3 relative."""
    mesh, U = _case("vortex")
    w = _weights(U.shape, 5)
    s = _solver(mesh)
    s.init_state(U)
    s.adjoint_record(2, checkpoint_every=2)
    g = s.adjoint_backward(w)
    rng = np.random.default_rng(6)

    def J(V):
        s.init_state(V)
        s.step(2)
        return float((w * s.get_state()).sum())

    for _ in range(3):
        v = rng.standard_normal(U.shape) * np.abs(U) * 1e-2
        eps = 1e-6
        fd = (J(U + eps * v) - J(U - eps * v)) / (2 * eps)
        ad = float((g * v).sum())
        assert abs(fd - ad) <= 1e-3 * max(abs(ad), 1e-3), (fd, ad)


def test_rollout_autograd_uses_adjoint_and_device_pointers():
    from paper_2007_00094_gb300.idp import rollout
    mesh, U = _case("sod")
    w = _weights(U.shape, 7)
    s = _solver(mesh)
    U0 = torch.as_tensor(U, device="cuda").requires_grad_(True)
    UN = rollout(s, U0, 3, checkpoint_every=2)
    J = (torch.as_tensor(w, device="cuda") * UN).sum()
    J.backward()
    s2 = _solver(mesh)
    s2.init_state(U)
    s2.adjoint_record(3, checkpoint_every=2)
    np.testing.assert_array_equal(UN.detach().cpu().numpy(), s2.get_state())
    g_host = s2.adjoint_backward(w)
    np.testing.assert_array_equal(U0.grad.cpu().numpy(), g_host)
    # device-pointer form of the single-stage adjoint equals the host form
    gd, td = s2.adjoint_euler_step(torch.as_tensor(U, device="cuda"), torch.as_tensor(w, device="cuda"))
    gh, th = s2.adjoint_euler_step(U, w)
    np.testing.assert_array_equal(gd.cpu().numpy(), gh)
    assert td == th


def test_adjoint_rejects_unsupported_configurations():
    from paper_2007_00094_gb300.idp import IdpError
    mesh, U = _case("wallbox")
    w = _weights(U.shape, 8)
    s = _solver(mesh)
    s.init_state(U)
    with pytest.raises(IdpError) as e:
        s.adjoint_backward(w)  # nothing recorded
    assert e.value.status == 9
    with pytest.raises(IdpError) as e:
        _solver(mesh, precision=1).adjoint_euler_step(U, w)
    assert e.value.status == 1
    with pytest.raises(IdpError) as e:
        _solver(mesh, limiter_passes=3).adjoint_euler_step(U, w)
    assert e.value.status == 1
    with pytest.raises(IdpError) as e:
        _solver(mesh, relax=1).adjoint_euler_step(U, w)
    assert e.value.status == 1
    with pytest.raises(IdpError) as e:
        s.adjoint_record(0)
    assert e.value.status == 1


def _box_pressure_case():
    from paper_2007_00094_gb300.objectives import BoxPressure
    mesh = W.vortex_mesh(16, jitter=0.2, seed=3)
    U = W.bumpy_vortex_state(mesh)
    s = _solver(mesh)
    return mesh, U, s, BoxPressure(mesh.x, s.matrices()[4])


def test_box_pressure_gradient_matches_reference_gradient():
    """The adjoint workload at reduced size (16^3 jittered periodic vortex with
    eight density bumps, J = sum_{x_i in [0.4,0.6]^3} m_i p_i after two
    SSP-RK3 steps) against torch.autograd through the PyTorch restatement.
    Measured: 2e-11 relative (2-norm) after 8 steps; the isentropic vortex
    keeps the limiter near its ill-conditioned point, where rounding of the
    traced values is amplified."""
    import oracle as O
    from oracle import torch_stage as T
    mesh, U, s, J = _box_pressure_case()
    s.init_state(U)
    s.adjoint_record(2, checkpoint_every=1)
    UN = s.get_state()
    g = s.adjoint_backward(J.gradient(UN))
    tm = T.TorchMesh(O.assemble(mesh))
    U0 = torch.as_tensor(U).clone().requires_grad_(True)
    V = U0
    for _ in range(2):
        V, _ = T.ssprk3_step(tm, V)
    (g_ref,) = torch.autograd.grad((torch.as_tensor(J.gradient(V.detach().numpy())) * V).sum(), (U0,))
    err = rel_field_err_l2(g, g_ref.numpy())
    assert err.max() <= 1e-9, err


def test_box_pressure_gradient_against_finite_differences():
    """The same workload over six steps (checkpoints every 5): the gradient
    against central differences of the CUDA forward run with eps = 1e-7
    (relative to the state) along 16 random directions and along 64 random
    single components.  The map is only piecewise smooth (limiter branches and
    Newton exits, min/max of bounds and wavespeeds, the CFL arg-min), and
    differences of that width cross branch points; measured errors stay below
    1e-2 of the largest directional derivative (directions) and of the largest
    gradient entry of the field (components), and shrink as eps does, while
    the adjoint itself matches the reference gradient to rounding."""
    mesh, U, s, J = _box_pressure_case()
    steps = 6
    s.init_state(U)
    s.adjoint_record(steps, checkpoint_every=5)
    g = s.adjoint_backward(J.gradient(s.get_state()))
    assert np.all(np.isfinite(g)) and np.abs(g).max() > 0.0

    def run(V):
        s.init_state(V)
        s.step(steps)
        return J(s.get_state())

    rng = np.random.default_rng(12)
    eps = 1e-7
    fd, ad = [], []
    for _ in range(16):
        v = rng.standard_normal(U.shape) * np.abs(U)
        fd.append((run(U + eps * v) - run(U - eps * v)) / (2 * eps))
        ad.append(float((g * v).sum()))
    fd, ad = np.array(fd), np.array(ad)
    assert np.abs(fd - ad).max() <= 1e-2 * np.abs(ad).max(), (fd, ad)
    gmax = np.abs(g).max(axis=1)
    for _ in range(64):
        f, i = int(rng.integers(5)), int(rng.integers(mesh.n_nodes))
        h = eps * max(abs(U[f, i]), 1e-3)
        Up, Um = U.copy(), U.copy()
        Up[f, i] += h
        Um[f, i] -= h
        d = (run(Up) - run(Um)) / (2 * h)
        assert abs(d - g[f, i]) <= 1e-2 * gmax[f], (f, i, d, g[f, i])

