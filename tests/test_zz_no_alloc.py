"""The allocation-free time-step bound against the context's own value.

idp_tau_max_noalloc serves callers that must not allocate device memory
themselves (a host framework that hands out all device memory from its own
pool, or a service that allocates only at start-up): it takes caller-owned
device arrays and keeps its scratch in a fixed device array of the library.
This test feeds it the matrices of a context (idp_get_matrices, also of a
context with renumbered rows) and the same state, and checks it against the
bound that idp_euler_step reports (IDP_FIELD_TAU_MAX), on two calls in a row
so that the scratch left by the first call cannot leak into the second; a
non-admissible state gives NaN.  The file sorts last so that a run stopping
at the first failure has run everything else.
"""
import numpy as np
import pytest

from gpu_common import require_gpu
from paper_2007_00094_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _cases():
    box = W.box_mesh((13, 11, 9), hi=(1.2, 1.0, 0.8), periodic=(False, False, False), jitter=0.25, seed=3)
    rho, u, p = W.vortex_primitive(box.x)
    Ubox = W.primitive_to_conserved(rho, u, p)
    Ubox[1:4] = np.where((box.bc & np.array([[1], [2], [4]])) > 0, 0.0, Ubox[1:4])
    ffs = W.forward_step_mesh(m=10, jitter=0.2, seed=2007)
    vortex = W.vortex_mesh(17)
    return [(box, Ubox), (ffs, W.forward_step_state(ffs)), (vortex, W.vortex_state(vortex))]


def test_noalloc_tau_max_matches_context():
    require_gpu()
    import torch

    from paper_2007_00094_gb300.idp import IDP_OK, Solver, idp_tau_max_noalloc

    for (mesh, U), renumber in [(c, 0) for c in _cases()] + [(_cases()[1], 1)]:
        s = Solver(mesh, renumber=renumber)
        s.init_state(U)
        s.euler_step(trace=True)
        ref = s.field("tau_max")
        rowptr, col, mij, cij, mi = s.matrices()
        dev = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda()
               for k, v in dict(rowptr=rowptr, col=col, cij=cij, mi=mi, U=U).items()}
        out = torch.empty(1, dtype=torch.float64, device="cuda")
        for call in range(2):
            out.fill_(float("nan"))
            st = idp_tau_max_noalloc(mesh.n_nodes, s.nnz, dev["rowptr"], dev["col"], dev["cij"], dev["mi"],
                                     dev["U"], out, torch.cuda.current_stream())
            assert st == IDP_OK
            torch.cuda.synchronize()
            got = float(out.item())
            assert abs(got - ref) <= 1e-14 * ref, (mesh.name, renumber, call, got, ref)
        s.close()


def test_noalloc_tau_max_is_nan_for_a_non_admissible_state():
    require_gpu()
    import torch

    from paper_2007_00094_gb300.idp import IDP_OK, Solver, idp_tau_max_noalloc

    mesh, U = _cases()[2]
    s = Solver(mesh)
    rowptr, col, mij, cij, mi = s.matrices()
    s.close()
    dev = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda()
           for k, v in dict(rowptr=rowptr, col=col, cij=cij, mi=mi).items()}
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    for bad in ("rho", "eps"):
        Ub = U.copy()
        k = mesh.n_nodes // 3
        if bad == "rho":
            Ub[0, k] = -0.5
        else:
            Ub[4, k] = 0.4 * 0.5 * (Ub[1:4, k] ** 2).sum() / Ub[0, k]  # epsilon < 0
        st = idp_tau_max_noalloc(mesh.n_nodes, cij.shape[1], dev["rowptr"], dev["col"], dev["cij"], dev["mi"],
                                 torch.from_numpy(Ub).cuda(), out, torch.cuda.current_stream())
        assert st == IDP_OK
        torch.cuda.synchronize()
        assert np.isnan(float(out.item())), bad


def test_noalloc_rejects_sizes_beyond_its_scratch():
    require_gpu()
    import torch

    from paper_2007_00094_gb300.idp import NOALLOC_MAX_NODES, idp_tau_max_noalloc

    buf = torch.zeros(8, dtype=torch.float64, device="cuda")
    assert idp_tau_max_noalloc(NOALLOC_MAX_NODES + 1, 1, buf, buf, buf, buf, buf, buf) == 1  # IDP_ERR_ARG
    assert idp_tau_max_noalloc(0, 1, buf, buf, buf, buf, buf, buf) == 1
