"""The differentiable PyTorch restatement of the stage (reference gradient of
the GPU adjoint) against the C oracle, and its gradient against central
finite differences of itself."""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import torch_stage as T
from paper_2007_00094_gb300 import workloads as W


def _case(name):
    if name == "vortex":
        m = W.vortex_mesh(7)
        return m, W.bumpy_vortex_state(m)
    if name == "wallbox":
        m = W.box_mesh((6, 5, 5), periodic=(False, False, False), jitter=0.2, seed=3)
        rho, u, p = W.vortex_primitive(m.x)
        U = W.primitive_to_conserved(rho, u, p)
        U[1:4] = np.where((m.bc & np.array([[1], [2], [4]])) > 0, 0.0, U[1:4])
        return m, U
    m = W.box_mesh((12, 3, 3), periodic=(False, True, True), jitter=0.1, seed=5)
    return m, W.sod_state(m)


@pytest.mark.parametrize("name", ["vortex", "wallbox", "sod"])
def test_torch_stage_matches_c_oracle(name):
    mesh, U = _case(name)
    om = O.assemble(mesh)
    tm = T.TorchMesh(om)
    ref, tau, st = O.ssprk3_step(om, U)
    assert st == 0
    out, tau_t = T.ssprk3_step(tm, torch.as_tensor(U))
    assert abs(float(tau_t) - tau) <= 1e-14 * tau
    scale = np.abs(ref).max()
    assert np.abs(out.numpy() - ref).max() <= 1e-12 * scale


def test_torch_gradient_against_finite_differences():
    """The stage is only piecewise smooth (limiter branches, min/max of the
    bounds, the p* branch), and central differences of width 2e-6 relative
    straddle some of the thousands of branch points of a coarse limited
    vortex; agreement is therefore checked to 1e-3 relative."""
    mesh, U = _case("vortex")
    om = O.assemble(mesh)
    tm = T.TorchMesh(om)
    U0 = torch.as_tensor(U).clone().requires_grad_(True)
    out, _ = T.ssprk3_step(tm, U0)
    w = torch.as_tensor(np.random.default_rng(0).normal(size=out.shape))
    J = (w * out).sum()
    (g,) = torch.autograd.grad(J, U0)
    rng = np.random.default_rng(1)
    for _ in range(3):
        v = torch.as_tensor(rng.normal(size=U.shape)) * torch.as_tensor(np.abs(U)) * 1e-2
        eps = 1e-6
        Jp = (w * T.ssprk3_step(tm, torch.as_tensor(U) + eps * v)[0]).sum()
        Jm = (w * T.ssprk3_step(tm, torch.as_tensor(U) - eps * v)[0]).sum()
        fd = float((Jp - Jm) / (2 * eps))
        ad = float((g * v).sum())
        assert abs(fd - ad) <= 1e-3 * max(abs(ad), 1e-3)


def test_torch_vjp_matches_jvp():
    """Reverse and forward mode agree to rounding on the branch taken."""
    mesh, U = _case("wallbox")
    om = O.assemble(mesh)
    tm = T.TorchMesh(om)
    U0 = torch.as_tensor(U)
    rng = np.random.default_rng(2)
    w = torch.as_tensor(rng.normal(size=U.shape))
    v = torch.as_tensor(rng.normal(size=U.shape)) * torch.abs(U0) * 1e-2

    def f(u):
        return T.euler_step(tm, u)[0]

    _, jv = torch.func.jvp(f, (U0,), (v,))
    _, vjp = torch.func.vjp(f, U0)
    (g,) = vjp(w)
    a, b = float((w * jv).sum()), float((g * v).sum())
    assert abs(a - b) <= 1e-12 * max(abs(a), 1.0)

