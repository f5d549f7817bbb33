"""Python access to the FP64 CPU oracle (oracle/idp_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of bench.py.  The product path (the CUDA library and its
binding) never imports this package.

The oracle restates Sec. 3 (Alg. 1-3) of Maier & Kronbichler, "Efficient
parallel 3D computation of the compressible Euler equations with an
invariant-domain preserving second-order finite-element scheme"
(arXiv:2007.00094) in plain C, FP64, one operation at a time.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "idp_oracle.c")
# IDP_ORACLE_LIB: load a prebuilt oracle library instead (the tests that plant
# mistakes in a copy of the source point it at the mutant's build)
_LIB_PATH = os.environ.get("IDP_ORACLE_LIB") or os.path.join(_HERE, "libidp_oracle.so")
_lib = None

_dp = C.POINTER(C.c_double)
_i64p = C.POINTER(C.c_int64)
_i32p = C.POINTER(C.c_int32)


class Params(C.Structure):
    _fields_ = [("gamma", C.c_double), ("cfl", C.c_double), ("limiter_passes", C.c_int),
                ("newton_max", C.c_int), ("newton_tol", C.c_double), ("newton_eps", C.c_double),
                ("n_threads", C.c_int), ("relax", C.c_int), ("psi_margin", C.c_double)]


def default_params(**kw) -> Params:
    """gamma = 7/5 (Sec. 2), c_cfl = 0.5, two limiter passes (Reading A16),
    two Newton steps and tolerance 1e-10 (Reading A11), eps = DBL_EPSILON
    (Reading A5), Psi margin 1e-13 (Reading A27)."""
    p = Params(gamma=1.4, cfl=0.5, limiter_passes=2, newton_max=2, newton_tol=1e-10,
               newton_eps=float(np.finfo(np.float64).eps), n_threads=1, relax=0, psi_margin=1e-13)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


class _Mesh(C.Structure):
    _fields_ = [("n", C.c_int64), ("rowptr", _i64p), ("col", _i64p), ("mij", _dp), ("cij", _dp),
                ("mi", _dp), ("bc", _i32p), ("inflow", _dp)]


class _Trace(C.Structure):
    _fields_ = [(name, _dp) for name in ("d", "alpha", "tau_max", "UL", "R", "bounds", "P", "l4", "U5",
                                         "l5", "Ulim")]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FP contraction, OpenMP over rows)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "idp_oracle.h"))):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off", "-fopenmp",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        L = _lib
        L.orc_sparsity.restype = C.c_int64
        L.orc_sparsity.argtypes = [C.c_int64, C.c_int64, _i64p, _i64p, _i64p]
        L.orc_assemble.restype = C.c_int
        L.orc_assemble.argtypes = [C.c_int64, C.c_int64, _i64p, _dp, _i64p, _i64p, _dp, _dp, _dp]
        L.orc_sparsity_nv.restype = C.c_int64
        L.orc_sparsity_nv.argtypes = [C.c_int64, C.c_int64, C.c_int, _i64p, _i64p, _i64p]
        L.orc_assemble_quad.restype = C.c_int
        L.orc_assemble_quad.argtypes = [C.c_int64, C.c_int64, _i64p, _dp, _i64p, _i64p, _dp, _dp, _dp]
        L.orc_node_quantities.restype = None
        L.orc_node_quantities.argtypes = [_dp, C.c_double, _dp]
        L.orc_lambda_max.restype = C.c_double
        L.orc_lambda_max.argtypes = [_dp, _dp, _dp, C.c_double]
        L.orc_limiter.restype = C.c_double
        L.orc_limiter.argtypes = [_dp, _dp, C.c_double, C.c_double, C.c_double, C.POINTER(Params)]
        L.orc_psi.restype = C.c_double
        L.orc_psi.argtypes = [_dp, C.c_double, C.c_double]
        L.orc_euler_step.restype = C.c_int
        L.orc_euler_step.argtypes = [C.POINTER(_Mesh), C.POINTER(Params), _dp, _dp, C.c_int, _dp,
                                     C.POINTER(_Trace)]
        L.orc_ssprk3_step.restype = C.c_int
        L.orc_ssprk3_step.argtypes = [C.POINTER(_Mesh), C.POINTER(Params), _dp, _dp]
        L.orc_ssprk3_step_fixed.restype = C.c_int
        L.orc_ssprk3_step_fixed.argtypes = [C.POINTER(_Mesh), C.POINTER(Params), _dp, C.c_double]
        L.orc_limiter_many.restype = None
        L.orc_limiter_many.argtypes = [C.c_int64, _dp, _dp, _dp, C.POINTER(Params), _dp, _i32p, _dp]
    return _lib


def _p(a, t=_dp):
    return a.ctypes.data_as(t)


@dataclass
class OracleMesh:
    """CSR matrices m_ij, c_ij, m_i assembled by the oracle from a HexMesh."""
    n: int
    rowptr: np.ndarray
    col: np.ndarray
    mij: np.ndarray
    cij: np.ndarray  # (3, nnz)
    mi: np.ndarray
    bc: np.ndarray
    inflow: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def struct(self) -> _Mesh:
        return _Mesh(self.n, _p(self.rowptr, _i64p), _p(self.col, _i64p), _p(self.mij), _p(self.cij),
                     _p(self.mi), _p(self.bc, _i32p), _p(self.inflow))

    def dense_row(self, i):
        a, b = self.rowptr[i], self.rowptr[i + 1]
        return self.col[a:b], self.mij[a:b], self.cij[:, a:b]


def assemble(mesh) -> OracleMesh:
    """Q1 matrices of Sec. 3.1 eq. (matrices) for ``mesh`` (a workloads.HexMesh of
    hexahedra, or of quadrilaterals when its cells have 4 vertices)."""
    L = lib()
    cells = np.ascontiguousarray(mesh.cells, dtype=np.int64)
    nv = cells.shape[1]
    if nv == 4:
        xyz = np.ascontiguousarray(mesh.cell_xyz[:, :, :2], dtype=np.float64)
        assemble_fn = L.orc_assemble_quad
    else:
        xyz = np.ascontiguousarray(mesh.cell_xyz, dtype=np.float64)
        assemble_fn = L.orc_assemble
    n = mesh.n_nodes
    rowptr = np.zeros(n + 1, dtype=np.int64)
    nnz = L.orc_sparsity_nv(n, cells.shape[0], nv, _p(cells, _i64p), _p(rowptr, _i64p), None)
    col = np.zeros(nnz, dtype=np.int64)
    L.orc_sparsity_nv(n, cells.shape[0], nv, _p(cells, _i64p), _p(rowptr, _i64p), _p(col, _i64p))
    mij = np.zeros(nnz)
    cij = np.zeros((3, nnz))
    mi = np.zeros(n)
    st = assemble_fn(n, cells.shape[0], _p(cells, _i64p), _p(xyz), _p(rowptr, _i64p), _p(col, _i64p),
                     _p(mij), _p(cij), _p(mi))
    if st != 0:
        raise ValueError("oracle assembly failed (inverted cell?)")
    inflow = np.zeros(5) if mesh.inflow is None else np.ascontiguousarray(mesh.inflow, dtype=np.float64)
    return OracleMesh(n, rowptr, col, mij, cij, mi, np.ascontiguousarray(mesh.bc, dtype=np.int32), inflow)


TRACE_SHAPES = {"d": "nnz", "alpha": "n", "tau_max": 1, "UL": "5n", "R": "5n", "bounds": "3n", "P": "5nnz",
                "l4": "nnz", "U5": "5n", "l5": "nnz", "Ulim": "5n"}


def euler_step(om: OracleMesh, U, tau=None, params=None, trace=False):
    """One euler_step (Alg. 1) with boundary post-processing.

    ``tau=None`` computes tau_n from the CFL condition (first RK stage);
    otherwise tau is fixed and checked (Reading A17).  Returns
    ``(U_out, tau, status, trace_dict)``.
    """
    prm = params or default_params()
    U = np.ascontiguousarray(U, dtype=np.float64)
    out = np.empty_like(U)
    t = C.c_double(0.0 if tau is None else float(tau))
    tr = None
    arrays = {}
    if trace:
        n, nnz = om.n, om.nnz
        size = {"nnz": nnz, "n": n, "5n": 5 * n, "3n": 3 * n, "5nnz": 5 * nnz, 1: 1}
        arrays = {k: np.zeros(size[v]) for k, v in TRACE_SHAPES.items()}
        tr = _Trace(**{k: _p(a) for k, a in arrays.items()})
    st = lib().orc_euler_step(C.byref(om.struct()), C.byref(prm), _p(U), C.byref(t), 0 if tau is None else 1,
                              _p(out), C.byref(tr) if tr is not None else None)
    if trace:
        n = om.n
        arrays["UL"] = arrays["UL"].reshape(5, n)
        arrays["R"] = arrays["R"].reshape(5, n)
        arrays["U5"] = arrays["U5"].reshape(5, n)
        arrays["Ulim"] = arrays["Ulim"].reshape(5, n)
        arrays["bounds"] = arrays["bounds"].reshape(3, n)
        arrays["P"] = arrays["P"].reshape(5, om.nnz)
        arrays["tau_max"] = float(arrays["tau_max"][0])
    return out, t.value, st, arrays


def ssprk3_step(om: OracleMesh, U, params=None):
    """One SSP-RK3 step (Sec. 3.6 eq. ssprk3); returns ``(U_new, tau, status)``."""
    prm = params or default_params()
    U = np.array(U, dtype=np.float64, order="C", copy=True)
    t = C.c_double(0.0)
    st = lib().orc_ssprk3_step(C.byref(om.struct()), C.byref(prm), _p(U), C.byref(t))
    return U, t.value, st


def ssprk3_step_fixed(om: OracleMesh, U, tau, params=None):
    """One SSP-RK3 step (eq. ssprk3) with a given tau_n for all three stages;
    returns ``(U_new, status)``."""
    prm = params or default_params()
    U = np.array(U, dtype=np.float64, order="C", copy=True)
    st = lib().orc_ssprk3_step_fixed(C.byref(om.struct()), C.byref(prm), _p(U), float(tau))
    return U, st


def run(om: OracleMesh, U, n_steps, params=None):
    """``n_steps`` SSP-RK3 steps; returns ``(U, t, taus)``."""
    t = 0.0
    taus = []
    for _ in range(n_steps):
        U, tau, st = ssprk3_step(om, U, params)
        if st != 0:
            raise RuntimeError(f"oracle step failed with status {st}")
        t += tau
        taus.append(tau)
    return U, t, taus


def lambda_max(n, Ui, Uj, gamma=1.4) -> float:
    """lambda~_max(n, U_i, U_j) of Sec. 3.7."""
    n = np.ascontiguousarray(n, dtype=np.float64)
    Ui = np.ascontiguousarray(Ui, dtype=np.float64)
    Uj = np.ascontiguousarray(Uj, dtype=np.float64)
    return lib().orc_lambda_max(_p(n), _p(Ui), _p(Uj), gamma)


def limiter(U, P, rho_min, rho_max, phi_min, params=None) -> float:
    """limiter.compute of Alg. 2."""
    prm = params or default_params()
    U = np.ascontiguousarray(U, dtype=np.float64)
    P = np.ascontiguousarray(P, dtype=np.float64)
    return lib().orc_limiter(_p(U), _p(P), rho_min, rho_max, phi_min, C.byref(prm))


def limiter_many(U, P, bounds, params=None):
    """limiter.compute of Alg. 2 for m independent calls: U, P of shape (5, m),
    bounds (3, m) = (rho_min, rho_max, phi_min).  Returns ``(t, hits, worst)``:
    the limiter values, the number of admissibility tests per call whose
    outcome the Psi margin decided (Reading A27) and the largest |Psi| / scale
    among them."""
    prm = params or default_params()
    U = np.ascontiguousarray(U, dtype=np.float64)
    P = np.ascontiguousarray(P, dtype=np.float64)
    bounds = np.ascontiguousarray(bounds, dtype=np.float64)
    m = U.shape[1]
    assert U.shape == (5, m) and P.shape == (5, m) and bounds.shape == (3, m)
    t = np.zeros(m)
    hits = np.zeros(m, dtype=np.int32)
    worst = np.zeros(m)
    lib().orc_limiter_many(m, _p(U), _p(P), _p(bounds), C.byref(prm), _p(t), _p(hits, _i32p), _p(worst))
    return t, hits, worst


def psi(U, phi_min, gamma=1.4) -> float:
    U = np.ascontiguousarray(U, dtype=np.float64)
    return lib().orc_psi(_p(U), phi_min, gamma)


def node_quantities(U, gamma=1.4):
    """(p, c, phi, eta, eta'(5)) of a single state (Sec. 2, Sec. 3.8)."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    out = np.zeros(9)
    lib().orc_node_quantities(_p(U), gamma, _p(out))
    return out
