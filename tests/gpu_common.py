"""Shared helpers of the GPU parity tests (test side only)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_00094_gb300 import build
    build.build()


def rel_field_err(a, b):
    """max_i |a - b| per field, relative to max_i |b| of that field; fields
    that vanish are measured against the largest field magnitude."""
    a = np.atleast_2d(a)
    b = np.atleast_2d(b)
    overall = np.abs(b).max()
    out = []
    for f in range(b.shape[0]):
        scale = np.abs(b[f]).max()
        if scale < 1e-12 * overall:
            scale = overall
        out.append(np.abs(a[f] - b[f]).max() / scale)
    return np.array(out)


def rel_field_err_l2(a, b):
    """||a_f - b_f||_2 / ||b_f||_2 per field (vanishing fields against the
    largest field norm)."""
    a = np.atleast_2d(a)
    b = np.atleast_2d(b)
    norms = np.sqrt((b * b).sum(axis=1))
    overall = norms.max()
    out = []
    for f in range(b.shape[0]):
        scale = norms[f] if norms[f] >= 1e-12 * overall else overall
        out.append(np.sqrt(((a[f] - b[f]) ** 2).sum()) / scale)
    return np.array(out)


def field_scales(b):
    """max_i |b_f| per field; fields that vanish take the largest field
    magnitude (the convention of rel_field_err)."""
    b = np.atleast_2d(b)
    sc = np.abs(b).max(axis=1)
    return np.where(sc < 1e-12 * sc.max(), sc.max(), sc)


def oracle_sensitivity(run, U, samples=8, rel=1e-15, seed=1):
    """How far the oracle's own results move when its input state is
    perturbed at rounding level: ``run(U)`` returns a dict of arrays (computed
    by the oracle only); each of ``samples`` seeded perturbations U (1 + rel
    xi), xi standard normal, is run as well, and the element-wise maximum
    deviation from the unperturbed results is returned per key (minus the
    size of the perturbation itself for state-shaped results).

    Isentropic data put the entropy limiter at its ill-conditioned point: phi
    is constant, Psi(t) along U + tP is flat near its root, and the root moves
    by far more than its inputs.  Two correct implementations that round
    differently then disagree at those nodes by about as much as the oracle
    disagrees with itself under a rounding-level perturbation of its input;
    this measures that allowance without using the CUDA path."""
    rng = np.random.default_rng(seed)
    base = run(U)
    spread = {k: np.zeros_like(v) for k, v in base.items()}
    for _ in range(samples):
        Up = U * (1.0 + rel * rng.standard_normal(U.shape))
        out = run(Up)
        for k, v in out.items():
            dev = np.abs(v - base[k])
            if v.shape == U.shape:
                dev = np.maximum(dev - np.abs(Up - U), 0.0)
            spread[k] = np.maximum(spread[k], dev)
    return base, spread
