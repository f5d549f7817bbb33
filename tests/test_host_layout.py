"""Host logic of the library without a GPU: the Q1 assembly and the sliced-ELL
layout (slice height 32) are built by the library's own host code
(csrc/idp_mesh.cpp, compiled here with g++ beside a small harness,
tests/host_layout.cpp) and checked for their invariants: every stored entry
has one slot in its row's lane, the transposed-slot map is an involution onto
the transposed entry, exactly one orientation of each pair is marked as the
one that evaluates the wavespeed (the row of the smaller caller id), one
diagonal per row, skew flags pairwise, columns in the library's numbering;
with reverse Cuthill-McKee renumbering the permutation is a bijection and
shrinks the bandwidth of a shuffled mesh."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2007_00094_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
_i64p = ctypes.POINTER(ctypes.c_int64)
_dp = ctypes.POINTER(ctypes.c_double)


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    out = str(tmp_path_factory.mktemp("host") / "libhost_layout.so")
    csrc = os.path.join(ROOT, "paper_2007_00094_gb300", "csrc")
    subprocess.run(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-fopenmp", "-I", os.path.join(ROOT, "include"),
                    "-I", csrc, "-o", out, os.path.join(ROOT, "tests", "host_layout.cpp"),
                    os.path.join(csrc, "idp_mesh.cpp")], check=True)
    lib = ctypes.CDLL(out)
    lib.host_layout.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int64, _i64p, _dp, ctypes.c_int, _i64p, _i64p]
    return lib


def _layout(lib, mesh, renumber):
    cells = np.ascontiguousarray(mesh.cells, dtype=np.int64)
    dim = mesh.dim
    xyz = np.ascontiguousarray(mesh.cell_xyz[:, :, :dim], dtype=np.float64)
    perm = np.zeros(mesh.n_nodes, dtype=np.int64)
    stats = np.zeros(9, dtype=np.int64)
    st = lib.host_layout(dim, mesh.n_nodes, cells.shape[0], cells.ctypes.data_as(_i64p), xyz.ctypes.data_as(_dp),
                         renumber, perm.ctypes.data_as(_i64p), stats.ctypes.data_as(_i64p))
    assert st == 0
    return perm, dict(zip(["n_slots", "perm", "tpos", "upper", "diag", "col", "skew", "map", "bandwidth"], stats))


def _shuffle(mesh, seed):
    p = np.random.default_rng(seed).permutation(mesh.n_nodes)
    inv = np.empty_like(p)
    inv[p] = np.arange(mesh.n_nodes)
    return W.HexMesh(x=mesh.x[inv], cells=p[mesh.cells], cell_xyz=mesh.cell_xyz, bc=mesh.bc[inv],
                     volume=mesh.volume, periodic=mesh.periodic)


MESHES = {
    "ffs10": lambda: W.forward_step_mesh(m=10, jitter=0.2, seed=2007),
    "periodic_box": lambda: W.box_mesh((9, 7, 5), periodic=(True, True, True), jitter=0.2, seed=2),
    "ffs2d": lambda: W.forward_step_mesh_2d(m=20, jitter=0.2, seed=3),
    "batch": lambda: W.concat_meshes([m for m, _ in W.random_riemann_batch(n_instances=3, side_range=(4, 7),
                                                                           seed=1)])[0],
}


@pytest.mark.parametrize("name", sorted(MESHES))
@pytest.mark.parametrize("renumber", [0, 1, 2])
def test_layout_invariants(harness, name, renumber):
    mesh = _shuffle(MESHES[name](), 7) if renumber else MESHES[name]()
    perm, s = _layout(harness, mesh, renumber)
    bad = {k: v for k, v in s.items() if k not in ("n_slots", "bandwidth") and v}
    assert not bad, bad
    assert sorted(perm) == list(range(mesh.n_nodes))
    if not renumber:
        np.testing.assert_array_equal(perm, np.arange(mesh.n_nodes))


@pytest.mark.parametrize("name", ["ffs10", "ffs2d"])
def test_renumbering_reduces_the_bandwidth_of_a_shuffled_mesh(harness, name):
    base = MESHES[name]()
    shuffled = _shuffle(base, 5)
    _, s_base = _layout(harness, base, 0)
    _, s_shuf = _layout(harness, shuffled, 0)
    _, s_rcm = _layout(harness, shuffled, 1)
    assert s_shuf["bandwidth"] > 0.8 * base.n_nodes  # a shuffle spreads neighbours over the whole range
    assert s_rcm["bandwidth"] <= 1.5 * s_base["bandwidth"]  # RCM brings it back to the structured order's scale


def _slice_spans(mesh, perm):
    """Mean number of distinct stencil nodes that the 32 rows of a slice
    touch (their gathers), for a row order perm (caller node -> row)."""
    import oracle as O

    om = O.assemble(mesh)
    rows_of = np.argsort(perm)  # caller node of each row
    spans = []
    for s0 in range(0, mesh.n_nodes - 31, 32):
        nodes = rows_of[s0:s0 + 32]
        cols = np.concatenate([om.col[om.rowptr[i]:om.rowptr[i + 1]] for i in nodes])
        spans.append(len(np.unique(cols)))
    return float(np.mean(spans))


def test_morton_order_depends_on_coordinates_only(harness):
    """renumber = 2 orders rows by the Morton key of the node coordinates: a
    shuffled copy of a mesh gets the same sequence of node positions."""
    base = MESHES["ffs10"]()
    shuf = _shuffle(base, 3)
    pb, _ = _layout(harness, base, 2)
    ps, _ = _layout(harness, shuf, 2)
    xb = np.empty_like(base.x)
    xb[pb] = base.x
    xs = np.empty_like(shuf.x)
    xs[ps] = shuf.x
    np.testing.assert_array_equal(xb, xs)


def test_morton_slices_are_compact_blocks(harness):
    """On a uniform box the 32 rows of a Morton slice are a 4 x 4 x 2 block:
    their stencils touch 6 x 6 x 4 = 144 nodes, where 32 consecutive rows of
    the lexicographic order (two x lines of 16) touch 18 x 4 x 3 = 216."""
    box = W.box_mesh((16, 16, 16), periodic=(False, False, False))
    p0, _ = _layout(harness, box, 0)
    p2, _ = _layout(harness, box, 2)
    lex, mor = _slice_spans(box, p0), _slice_spans(box, p2)
    assert mor < 0.8 * lex, (mor, lex)
