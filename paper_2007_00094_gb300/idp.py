"""Thin ctypes binding of libidp (include/idp.h).

Argument marshalling only: every step of the stage runs in the CUDA kernels
of libidp.so.  Functions keep the C names (``idp_create``, ``idp_step``, ...);
:class:`Solver` bundles them for convenience.  Device buffers may be torch
CUDA tensors (their ``data_ptr()`` is passed with ``on_device=1``), streams
may be ``torch.cuda.Stream`` objects or raw ``cudaStream_t`` integers.

If libidp.so has not been built (``python -m paper_2007_00094_gb300.build``)
loading fails with an ImportError: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libidp.so")

IDP_OK = 0
IDP_ERR_ARG, IDP_ERR_BOUNDS = 1, 7
STATUS_NAMES = {0: "IDP_OK", 1: "IDP_ERR_ARG", 2: "IDP_ERR_CUDA", 3: "IDP_ERR_OOM", 4: "IDP_ERR_STATE_NOT_ADMISSIBLE",
                5: "IDP_ERR_CFL", 6: "IDP_ERR_NONFINITE", 7: "IDP_ERR_BOUNDS", 8: "IDP_ERR_TIMEOUT",
                9: "IDP_ERR_STATE"}
FIELDS = {"d": 0, "alpha": 1, "UL": 2, "R": 3, "bounds": 4, "P": 5, "l4": 6, "U5": 7, "l5": 8, "Ulim": 9,
          "tau_max": 10}

# Every symbol include/idp.h declares.
EXPORTED = ["idp_config_default", "idp_create", "idp_destroy", "idp_last_error", "idp_status_string",
            "idp_upload_mesh_hex", "idp_mesh_info", "idp_get_matrices", "idp_init_state", "idp_get_state",
            "idp_step", "idp_euler_step", "idp_synchronize", "idp_get_time", "idp_set_time", "idp_get_field",
            "idp_check_bounds", "idp_launch_count", "idp_profile", "idp_profile_read", "idp_tau_max_noalloc", "idp_set_instances",
            "idp_get_instance_times", "idp_set_schedule", "idp_autotune", "idp_adjoint_euler_step",
            "idp_adjoint_record", "idp_adjoint_backward", "idp_barrier_selftest", "idp_upload_mesh_quad",
            "idp_entry_table_size", "idp_upload_sparsity", "idp_check_local_bounds", "idp_probe_fp64_peak",
            "idp_row_pattern_count", "idp_shard_plan_create", "idp_shard_plan_destroy", "idp_shard_plan_info",
            "idp_shard_plan_nodes", "idp_shard_plan_csr", "idp_shard_plan_list", "idp_shards_create",
            "idp_shards_destroy", "idp_shards_last_error", "idp_shards_init_state", "idp_shards_get_state",
            "idp_shards_step", "idp_shards_synchronize", "idp_shards_get_time", "idp_shards_context",
            "idp_shards_halo_size"]
SEND_NODES, RECV_NODES, SEND_ENTRIES, RECV_ENTRIES = 0, 1, 2, 3
NOALLOC_MAX_NODES = 2097152
KERNELS = ["node", "edge", "diag", "low_order", "flux_limit", "limiter_pass", "final", "adj_final", "adj_pass",
           "adj_flux", "adj_low", "adj_tau", "adj_diag", "adj_edge", "adj_gather"]


class IdpConfig(C.Structure):
    _fields_ = [("gamma", C.c_double), ("cfl", C.c_double), ("limiter_passes", C.c_int), ("newton_max", C.c_int),
                ("newton_tol", C.c_double), ("newton_eps", C.c_double), ("precision", C.c_int),
                ("schedule", C.c_int), ("barrier_spin_limit", C.c_int64), ("relax", C.c_int),
                ("entry_table", C.c_int), ("adjoint_store_stages", C.c_int), ("renumber", C.c_int)]


class BoundsReport(C.Structure):
    _fields_ = [("n_rho_nonpositive", C.c_int64), ("n_eps_nonpositive", C.c_int64), ("n_nonfinite", C.c_int64),
                ("rho_min", C.c_double), ("eps_min", C.c_double), ("n_bound_rows", C.c_int64),
                ("n_rho_below_min", C.c_int64), ("n_rho_above_max", C.c_int64), ("n_phi_below_min", C.c_int64),
                ("rho_min_violation", C.c_double), ("rho_max_violation", C.c_double),
                ("phi_min_violation", C.c_double), ("slack_rho", C.c_double), ("slack_phi", C.c_double)]


class IdpError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lib = None
_vp = C.c_void_p
_dp = C.POINTER(C.c_double)
_i64p = C.POINTER(C.c_int64)
_i32p = C.POINTER(C.c_int32)


def load(path: str = LIB_PATH):
    """Loads libidp.so (raises ImportError when it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libidp.so not built at {path}; run paper_2007_00094_gb300.build.build()")
    L = C.CDLL(path)
    L.idp_config_default.argtypes = [C.POINTER(IdpConfig)]
    L.idp_config_default.restype = None
    L.idp_create.argtypes = [C.POINTER(IdpConfig), _vp, C.POINTER(_vp)]
    L.idp_destroy.argtypes = [_vp]
    L.idp_destroy.restype = None
    L.idp_last_error.argtypes = [_vp]
    L.idp_last_error.restype = C.c_char_p
    L.idp_status_string.argtypes = [C.c_int]
    L.idp_status_string.restype = C.c_char_p
    L.idp_upload_mesh_hex.argtypes = [_vp, C.c_int64, C.c_int64, _i64p, _dp, _i32p, _dp]
    L.idp_upload_mesh_quad.argtypes = [_vp, C.c_int64, C.c_int64, _i64p, _dp, _i32p, _dp]
    L.idp_upload_sparsity.argtypes = [_vp, C.c_int64, _i64p, _i64p, _dp, _dp, _dp, _i32p, _dp]
    L.idp_mesh_info.argtypes = [_vp, _i64p, _i64p]
    L.idp_entry_table_size.argtypes = [_vp, _i64p]
    L.idp_row_pattern_count.argtypes = [_vp, _i64p]
    L.idp_get_matrices.argtypes = [_vp, _i64p, _i64p, _dp, _dp, _dp]
    L.idp_init_state.argtypes = [_vp, _vp, C.c_int]
    L.idp_get_state.argtypes = [_vp, _vp, C.c_int]
    L.idp_step.argtypes = [_vp, C.c_int]
    L.idp_euler_step.argtypes = [_vp, C.c_double, C.c_int, _dp]
    L.idp_synchronize.argtypes = [_vp]
    L.idp_get_time.argtypes = [_vp, _dp, _dp]
    L.idp_set_time.argtypes = [_vp, C.c_double]
    L.idp_get_field.argtypes = [_vp, C.c_int, _dp]
    L.idp_check_bounds.argtypes = [_vp, C.POINTER(BoundsReport)]
    L.idp_check_local_bounds.argtypes = [_vp, _vp, _vp, C.c_int, C.POINTER(BoundsReport)]
    L.idp_launch_count.argtypes = [_vp]
    L.idp_launch_count.restype = C.c_int64
    L.idp_profile.argtypes = [_vp, C.c_int]
    L.idp_profile_read.argtypes = [_vp, _dp, _i64p]
    L.idp_tau_max_noalloc.argtypes = [C.c_int64, C.c_int64, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
    L.idp_probe_fp64_peak.argtypes = [_vp, C.c_int64, _dp, _dp]
    L.idp_set_instances.argtypes = [_vp, C.c_int64, _i64p]
    L.idp_get_instance_times.argtypes = [_vp, _dp, _dp]
    L.idp_set_schedule.argtypes = [_vp, C.c_int, C.c_int, C.c_int]
    L.idp_autotune.argtypes = [_vp, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int), _dp]
    L.idp_adjoint_euler_step.argtypes = [_vp, _vp, C.c_double, _vp, _vp, _dp, C.c_int]
    L.idp_adjoint_record.argtypes = [_vp, C.c_int, C.c_int]
    L.idp_adjoint_backward.argtypes = [_vp, _vp, _vp, C.c_int]
    L.idp_barrier_selftest.argtypes = [_vp, C.c_int, C.c_int, C.c_int, C.c_longlong, C.POINTER(C.c_int)]
    L.idp_shard_plan_create.argtypes = [C.c_int64, _i64p, _i64p, C.c_int, _i64p, C.POINTER(_vp)]
    L.idp_shard_plan_destroy.argtypes = [_vp]
    L.idp_shard_plan_destroy.restype = None
    L.idp_shard_plan_info.argtypes = [_vp, C.c_int, _i64p, _i64p, _i64p, _i64p]
    L.idp_shard_plan_nodes.argtypes = [_vp, C.c_int, _i64p]
    L.idp_shard_plan_csr.argtypes = [_vp, C.c_int, _i64p, _i64p, _i64p]
    L.idp_shard_plan_list.argtypes = [_vp, C.c_int, C.c_int, C.c_int, _i64p, _i64p]
    L.idp_shards_create.argtypes = [C.POINTER(IdpConfig), _vp, _vp, _dp, _dp, _dp, _i32p, _dp, C.POINTER(_vp)]
    L.idp_shards_destroy.argtypes = [_vp]
    L.idp_shards_destroy.restype = None
    L.idp_shards_last_error.argtypes = [_vp]
    L.idp_shards_last_error.restype = C.c_char_p
    L.idp_shards_init_state.argtypes = [_vp, _dp]
    L.idp_shards_get_state.argtypes = [_vp, _dp]
    L.idp_shards_step.argtypes = [_vp, C.c_int]
    L.idp_shards_synchronize.argtypes = [_vp]
    L.idp_shards_get_time.argtypes = [_vp, _dp, _dp]
    L.idp_shards_context.argtypes = [_vp, C.c_int, C.POINTER(_vp)]
    L.idp_shards_halo_size.argtypes = [_vp, _i64p, _i64p, _i64p]
    _lib = L
    return L


def idp_tau_max_noalloc(n_nodes, nnz, rowptr, col, cij, mi, U, tau_max, stream=None):
    """tau_max = min_i m_i/(-2 d_ii) from caller-owned device arrays, without
    any device allocation (see include/idp.h).  Array arguments are device
    pointers (ints) or CUDA tensors; returns the idp_status code."""
    ptrs = [a.data_ptr() if hasattr(a, "data_ptr") else int(a) for a in (rowptr, col, cij, mi, U, tau_max)]
    return load().idp_tau_max_noalloc(int(n_nodes), int(nnz), *ptrs, _stream_handle(stream))


def idp_probe_fp64_peak(fma_per_thread=1 << 18, stream=None):
    """Measured FP64 FMA rate of the current GPU: (TFLOP/s, ms)."""
    tf, ms = C.c_double(), C.c_double()
    st = load().idp_probe_fp64_peak(_stream_handle(stream), int(fma_per_thread), C.byref(tf), C.byref(ms))
    if st != IDP_OK:
        raise IdpError(st, "idp_probe_fp64_peak failed")
    return tf.value, ms.value


def _ptr(a, t=_dp):
    return a.ctypes.data_as(t)


def _stream_handle(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def idp_config_default() -> IdpConfig:
    cfg = IdpConfig()
    load().idp_config_default(C.byref(cfg))
    return cfg


def _check(ctx, st):
    if st != IDP_OK:
        msg = load().idp_last_error(ctx).decode() if ctx else ""
        raise IdpError(st, msg)


class Solver:
    """One libidp context: a mesh, its matrices and the stage buffers."""

    def __init__(self, mesh=None, config: IdpConfig | None = None, stream=None, sparsity=None, **overrides):
        """``mesh``: a workloads.HexMesh (hexahedra or quadrilaterals), uploaded
        with idp_upload_mesh_hex/quad; or ``sparsity``: pre-assembled matrices
        with attributes (or keys) rowptr, col, mij, cij (3, nnz), mi (or None),
        bc (or None), inflow (or None), uploaded with idp_upload_sparsity."""
        L = load()
        cfg = config or idp_config_default()
        for k, v in overrides.items():
            setattr(cfg, k, v)
        self.config = cfg
        self._ctx = _vp()
        st = L.idp_create(C.byref(cfg), _stream_handle(stream), C.byref(self._ctx))
        if st != IDP_OK:
            raise IdpError(st, "idp_create failed")
        if sparsity is not None:
            self._upload_sparsity(sparsity)
            return
        self.n = mesh.n_nodes
        cells = np.ascontiguousarray(mesh.cells, dtype=np.int64)
        bc = np.ascontiguousarray(mesh.bc, dtype=np.int32)
        inflow = None if mesh.inflow is None else np.ascontiguousarray(mesh.inflow, dtype=np.float64)
        if cells.shape[1] == 4:  # Q1 quadrilaterals (2D)
            xyz = np.ascontiguousarray(mesh.cell_xyz[:, :, :2], dtype=np.float64)
            upload = L.idp_upload_mesh_quad
        else:
            xyz = np.ascontiguousarray(mesh.cell_xyz, dtype=np.float64)
            upload = L.idp_upload_mesh_hex
        _check(self._ctx, upload(self._ctx, mesh.n_nodes, cells.shape[0], _ptr(cells, _i64p), _ptr(xyz),
                                 _ptr(bc, _i32p), None if inflow is None else _ptr(inflow)))
        n, nnz = C.c_int64(), C.c_int64()
        _check(self._ctx, L.idp_mesh_info(self._ctx, C.byref(n), C.byref(nnz)))
        self.nnz = nnz.value

    def _upload_sparsity(self, sp):
        get = (lambda k: sp.get(k)) if isinstance(sp, dict) else (lambda k: getattr(sp, k, None))
        rowptr = np.ascontiguousarray(get("rowptr"), dtype=np.int64)
        col = np.ascontiguousarray(get("col"), dtype=np.int64)
        mij = np.ascontiguousarray(get("mij"), dtype=np.float64)
        cij = np.ascontiguousarray(get("cij"), dtype=np.float64)
        mi, bc, inflow = get("mi"), get("bc"), get("inflow")
        mi = None if mi is None else np.ascontiguousarray(mi, dtype=np.float64)
        bc = None if bc is None else np.ascontiguousarray(bc, dtype=np.int32)
        inflow = None if inflow is None else np.ascontiguousarray(inflow, dtype=np.float64)
        self.n = len(rowptr) - 1
        assert cij.shape == (3, len(col)) and mij.shape == (len(col),)
        _check(self._ctx, load().idp_upload_sparsity(
            self._ctx, self.n, _ptr(rowptr, _i64p), _ptr(col, _i64p), _ptr(mij), _ptr(cij),
            None if mi is None else _ptr(mi), None if bc is None else _ptr(bc, _i32p),
            None if inflow is None else _ptr(inflow)))
        n, nnz = C.c_int64(), C.c_int64()
        _check(self._ctx, load().idp_mesh_info(self._ctx, C.byref(n), C.byref(nnz)))
        self.nnz = nnz.value

    def close(self):
        if self._ctx:
            load().idp_destroy(self._ctx)
            self._ctx = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_state(self, U):
        """U: (5, n) float64 numpy array or CUDA torch tensor (caller order)."""
        if hasattr(U, "data_ptr"):
            assert U.is_cuda and U.dtype.itemsize == 8 and U.is_contiguous() and U.numel() == 5 * self.n
            _check(self._ctx, load().idp_init_state(self._ctx, U.data_ptr(), 1))
        else:
            a = np.ascontiguousarray(U, dtype=np.float64)
            assert a.size == 5 * self.n
            _check(self._ctx, load().idp_init_state(self._ctx, a.ctypes.data, 0))

    def get_state(self, out=None):
        if out is not None and hasattr(out, "data_ptr"):
            _check(self._ctx, load().idp_get_state(self._ctx, out.data_ptr(), 1))
            return out
        a = np.empty((5, self.n)) if out is None else out
        _check(self._ctx, load().idp_get_state(self._ctx, a.ctypes.data, 0))
        return a

    def step(self, n_steps=1):
        """Enqueues n_steps SSP-RK3 steps (no host synchronisation)."""
        _check(self._ctx, load().idp_step(self._ctx, int(n_steps)))

    def synchronize(self):
        _check(self._ctx, load().idp_synchronize(self._ctx))

    def euler_step(self, tau=None, trace=False):
        """One euler_step in place; returns tau."""
        t = C.c_double(0.0)
        _check(self._ctx, load().idp_euler_step(self._ctx, 0.0 if tau is None else float(tau), int(trace),
                                                C.byref(t)))
        return t.value

    def field(self, name):
        which = FIELDS[name]
        size = {"d": self.nnz, "alpha": self.n, "UL": 5 * self.n, "R": 5 * self.n, "bounds": 3 * self.n,
                "P": 5 * self.nnz, "l4": self.nnz, "U5": 5 * self.n, "l5": self.nnz, "Ulim": 5 * self.n,
                "tau_max": 1}[name]
        out = np.empty(size)
        _check(self._ctx, load().idp_get_field(self._ctx, which, _ptr(out)))
        shapes = {"UL": (5, self.n), "R": (5, self.n), "bounds": (3, self.n), "P": (5, self.nnz),
                  "U5": (5, self.n), "Ulim": (5, self.n)}
        if name == "tau_max":
            return float(out[0])
        return out.reshape(shapes[name]) if name in shapes else out

    def entry_table_size(self) -> int:
        """Distinct FP32 entries in the mixed stage's entry table (0: per-entry arrays)."""
        v = C.c_int64(0)
        _check(self._ctx, load().idp_entry_table_size(self._ctx, C.byref(v)))
        return int(v.value)

    def row_pattern_count(self) -> int:
        """Row patterns of the mixed stage (0: per-entry column and transpose arrays)."""
        v = C.c_int64(0)
        _check(self._ctx, load().idp_row_pattern_count(self._ctx, C.byref(v)))
        return int(v.value)

    def matrices(self):
        n, nnz = self.n, self.nnz
        rowptr = np.empty(n + 1, dtype=np.int64)
        col = np.empty(nnz, dtype=np.int64)
        mij = np.empty(nnz)
        cij = np.empty((3, nnz))
        mi = np.empty(n)
        _check(self._ctx, load().idp_get_matrices(self._ctx, _ptr(rowptr, _i64p), _ptr(col, _i64p), _ptr(mij),
                                                  _ptr(cij), _ptr(mi)))
        return rowptr, col, mij, cij, mi

    def time(self):
        t, tau = C.c_double(), C.c_double()
        _check(self._ctx, load().idp_get_time(self._ctx, C.byref(t), C.byref(tau)))
        return t.value, tau.value

    def set_time(self, t):
        _check(self._ctx, load().idp_set_time(self._ctx, float(t)))

    def check_bounds(self):
        """idp_check_bounds: (status, BoundsReport) for the current state and
        the last stage's local bounds."""
        rep = BoundsReport()
        st = load().idp_check_bounds(self._ctx, C.byref(rep))
        return st, rep

    def check_local_bounds(self, U, bounds):
        """idp_check_local_bounds of a (5, n) state against (3, n) bounds
        (numpy arrays, caller order); returns (status, BoundsReport)."""
        U = np.ascontiguousarray(U, dtype=np.float64)
        bounds = np.ascontiguousarray(bounds, dtype=np.float64)
        assert U.shape == (5, self.n) and bounds.shape == (3, self.n)
        rep = BoundsReport()
        st = load().idp_check_local_bounds(self._ctx, U.ctypes.data, bounds.ctypes.data, 0, C.byref(rep))
        return st, rep

    def launch_count(self):
        return load().idp_launch_count(self._ctx)

    def profile(self, enable=True):
        """Starts (clearing earlier records) or stops per-kernel event timing."""
        _check(self._ctx, load().idp_profile(self._ctx, int(enable)))

    def profile_read(self):
        """{kernel: (milliseconds, launches)} since profiling started."""
        ms = np.zeros(len(KERNELS))
        cnt = np.zeros(len(KERNELS), dtype=np.int64)
        _check(self._ctx, load().idp_profile_read(self._ctx, _ptr(ms), _ptr(cnt, _i64p)))
        return {k: (float(ms[q]), int(cnt[q])) for q, k in enumerate(KERNELS)}

    def set_instances(self, node_offsets):
        """Declares independent instances by contiguous node ranges."""
        off = np.ascontiguousarray(node_offsets, dtype=np.int64)
        _check(self._ctx, load().idp_set_instances(self._ctx, len(off) - 1, _ptr(off, _i64p)))
        self.n_instances = len(off) - 1

    def instance_times(self):
        k = getattr(self, "n_instances", 1)
        t, tau = np.zeros(k), np.zeros(k)
        _check(self._ctx, load().idp_get_instance_times(self._ctx, _ptr(t), _ptr(tau)))
        return t, tau

    def set_schedule(self, block_size=128, use_graph=False, persistent=False):
        _check(self._ctx, load().idp_set_schedule(self._ctx, int(block_size), int(bool(use_graph)),
                                                  int(bool(persistent))))

    def autotune(self, steps=2):
        """Times every schedule and keeps the fastest; returns
        (block, graph, persistent, ms/step)."""
        b, g, p, ms = C.c_int(), C.c_int(), C.c_int(), C.c_double()
        _check(self._ctx, load().idp_autotune(self._ctx, int(steps), C.byref(b), C.byref(g), C.byref(p),
                                              C.byref(ms)))
        return b.value, bool(g.value), bool(p.value), ms.value

    def barrier_selftest(self, blocks, rounds, skip_block0=False, spin_limit=1 << 20):
        """Runs the grid-barrier self-test; returns (status, block-passes)."""
        passes = C.c_int(0)
        st = load().idp_barrier_selftest(self._ctx, int(blocks), int(rounds), int(bool(skip_block0)),
                                         int(spin_limit), C.byref(passes))
        return st, passes.value

    # -- reverse mode ---------------------------------------------------------

    def _arrays(self, *arrays):
        """Pointers of (5, n) float64 arrays: all CUDA tensors (on_device=1)
        or all numpy arrays (on_device=0)."""
        dev = hasattr(arrays[0], "data_ptr")
        ptrs = []
        for a in arrays:
            if dev:
                assert a.is_cuda and a.dtype.itemsize == 8 and a.is_contiguous() and a.numel() == 5 * self.n
                ptrs.append(a.data_ptr())
            else:
                assert a.dtype == np.float64 and a.flags.c_contiguous and a.size == 5 * self.n
                ptrs.append(a.ctypes.data)
        return ptrs, int(dev)

    def adjoint_euler_step(self, U, gE, tau=None, out=None):
        """Adjoint of one euler_step at input U for the output adjoint gE;
        returns (gU, dJ/dtau).  tau=None: tau_n computed from U."""
        if out is None:
            out = gE.new_empty(gE.shape) if hasattr(gE, "data_ptr") else np.empty((5, self.n))
        if not hasattr(U, "data_ptr"):
            U = np.ascontiguousarray(U, dtype=np.float64)
            gE = np.ascontiguousarray(gE, dtype=np.float64)
        (pu, pg, po), dev = self._arrays(U, gE, out)
        gt = C.c_double(0.0)
        _check(self._ctx, load().idp_adjoint_euler_step(self._ctx, pu, 0.0 if tau is None else float(tau), pg, po,
                                                        C.byref(gt), dev))
        return out, gt.value

    def adjoint_record(self, n_steps, checkpoint_every=10):
        """Advances n_steps SSP-RK3 steps, keeping checkpoints for adjoint_backward."""
        _check(self._ctx, load().idp_adjoint_record(self._ctx, int(n_steps), int(checkpoint_every)))

    def adjoint_backward(self, gU_final, out=None):
        """Adjoint of the recorded run's initial state for the final-state adjoint gU_final."""
        if out is None:
            out = gU_final.new_empty(gU_final.shape) if hasattr(gU_final, "data_ptr") else np.empty((5, self.n))
        if not hasattr(gU_final, "data_ptr"):
            gU_final = np.ascontiguousarray(gU_final, dtype=np.float64)
        (pg, po), dev = self._arrays(gU_final, out)
        _check(self._ctx, load().idp_adjoint_backward(self._ctx, pg, po, dev))
        return out


def _rollout_function():
    import torch

    class Rollout(torch.autograd.Function):
        """U^N(U^0) of n_steps SSP-RK3 steps; backward runs the library's adjoint."""

        @staticmethod
        def forward(ctx, U0, solver, n_steps, checkpoint_every):
            solver.init_state(U0.detach().contiguous())
            solver.adjoint_record(n_steps, checkpoint_every)
            ctx.solver = solver
            return solver.get_state(torch.empty_like(U0))

        @staticmethod
        def backward(ctx, g):
            return ctx.solver.adjoint_backward(g.contiguous()), None, None, None

    return Rollout


_ROLLOUT = None


def rollout(solver, U0, n_steps, checkpoint_every=10):
    """Differentiable run of n_steps SSP-RK3 steps from U0 (a (5, n) float64
    CUDA tensor): returns U^N; torch.autograd gradients flow back through the
    discrete adjoint (idp_adjoint_record / idp_adjoint_backward)."""
    global _ROLLOUT
    if _ROLLOUT is None:
        _ROLLOUT = _rollout_function()
    return _ROLLOUT.apply(U0, solver, int(n_steps), int(checkpoint_every))


class ShardPlan:
    """Row partition with one ghost layer and its exchange lists
    (idp_shard_plan_*; host memory only, usable without a GPU)."""

    def __init__(self, rowptr, col, n_shards, row_begin=None):
        L = load()
        self.rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
        self.col = np.ascontiguousarray(col, dtype=np.int64)
        self.n = len(self.rowptr) - 1
        self.n_shards = int(n_shards)
        rb = None if row_begin is None else np.ascontiguousarray(row_begin, dtype=np.int64)
        self._plan = _vp()
        st = L.idp_shard_plan_create(self.n, _ptr(self.rowptr, _i64p), _ptr(self.col, _i64p), self.n_shards,
                                     None if rb is None else _ptr(rb, _i64p), C.byref(self._plan))
        if st != IDP_OK:
            raise IdpError(st, "idp_shard_plan_create failed")

    def close(self):
        if self._plan:
            load().idp_shard_plan_destroy(self._plan)
            self._plan = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self, shard):
        """(n_local, own_begin, own_end, nnz_local) of one shard."""
        v = [C.c_int64() for _ in range(4)]
        st = load().idp_shard_plan_info(self._plan, int(shard), *[C.byref(x) for x in v])
        if st != IDP_OK:
            raise IdpError(st, "idp_shard_plan_info failed")
        return tuple(int(x.value) for x in v)

    def nodes(self, shard):
        out = np.empty(self.info(shard)[0], dtype=np.int64)
        _check(None, load().idp_shard_plan_nodes(self._plan, int(shard), _ptr(out, _i64p)))
        return out

    def csr(self, shard):
        """Local (rowptr, col, global entry of each local entry)."""
        nl, _, _, el = self.info(shard)
        rp, cl, en = np.empty(nl + 1, np.int64), np.empty(el, np.int64), np.empty(el, np.int64)
        _check(None, load().idp_shard_plan_csr(self._plan, int(shard), _ptr(rp, _i64p), _ptr(cl, _i64p),
                                               _ptr(en, _i64p)))
        return rp, cl, en

    def list(self, shard, peer, kind):
        """Exchange list (SEND_NODES, RECV_NODES, SEND_ENTRIES, RECV_ENTRIES) of shard for peer."""
        cnt = C.c_int64()
        L = load()
        _check(None, L.idp_shard_plan_list(self._plan, int(shard), int(peer), int(kind), C.byref(cnt), None))
        out = np.empty(cnt.value, dtype=np.int64)
        if cnt.value:
            _check(None, L.idp_shard_plan_list(self._plan, int(shard), int(peer), int(kind), C.byref(cnt),
                                               _ptr(out, _i64p)))
        return out


class ShardedSolver:
    """The sharded stage on the current GPU (idp_shards_*): one context per
    shard of a ShardPlan, with halo exchanges between the stage's phases."""

    def __init__(self, sparsity, n_shards=2, row_begin=None, config: IdpConfig | None = None, stream=None,
                 **overrides):
        """``sparsity``: the whole mesh's matrices as for Solver(sparsity=...)
        (rowptr, col, mij, cij (3, nnz), mi, bc, inflow)."""
        L = load()
        get = (lambda k: sparsity.get(k)) if isinstance(sparsity, dict) else (lambda k: getattr(sparsity, k, None))
        self.plan = ShardPlan(get("rowptr"), get("col"), n_shards, row_begin)
        self.n = self.plan.n
        cfg = config or idp_config_default()
        for k, v in overrides.items():
            setattr(cfg, k, v)
        self.config = cfg
        mij = np.ascontiguousarray(get("mij"), dtype=np.float64)
        cij = np.ascontiguousarray(get("cij"), dtype=np.float64)
        mi, bc, inflow = get("mi"), get("bc"), get("inflow")
        mi = None if mi is None else np.ascontiguousarray(mi, dtype=np.float64)
        bc = None if bc is None else np.ascontiguousarray(bc, dtype=np.int32)
        inflow = None if inflow is None else np.ascontiguousarray(inflow, dtype=np.float64)
        assert cij.shape == (3, len(self.plan.col)) and mij.shape == (len(self.plan.col),)
        self._sh = _vp()
        st = L.idp_shards_create(C.byref(cfg), _stream_handle(stream), self.plan._plan, _ptr(mij), _ptr(cij),
                                 None if mi is None else _ptr(mi), None if bc is None else _ptr(bc, _i32p),
                                 None if inflow is None else _ptr(inflow), C.byref(self._sh))
        if st != IDP_OK:
            raise IdpError(st, "idp_shards_create failed")

    def _check(self, st):
        if st != IDP_OK:
            raise IdpError(st, load().idp_shards_last_error(self._sh).decode())

    def close(self):
        if self._sh:
            load().idp_shards_destroy(self._sh)
            self._sh = _vp()
        self.plan.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_state(self, U):
        a = np.ascontiguousarray(U, dtype=np.float64)
        assert a.size == 5 * self.n
        self._check(load().idp_shards_init_state(self._sh, _ptr(a)))

    def get_state(self):
        a = np.empty((5, self.n))
        self._check(load().idp_shards_get_state(self._sh, _ptr(a)))
        return a

    def step(self, n_steps=1):
        self._check(load().idp_shards_step(self._sh, int(n_steps)))

    def synchronize(self):
        self._check(load().idp_shards_synchronize(self._sh))

    def time(self):
        t, tau = C.c_double(), C.c_double()
        self._check(load().idp_shards_get_time(self._sh, C.byref(t), C.byref(tau)))
        return t.value, tau.value

    def halo_size(self):
        """(node values per field, entry values) per exchange, and the launches of the last step call."""
        a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
        self._check(load().idp_shards_halo_size(self._sh, C.byref(a), C.byref(b), C.byref(c)))
        return int(a.value), int(b.value), int(c.value)
