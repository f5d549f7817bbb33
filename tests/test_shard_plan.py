"""Row partition with one ghost layer and its exchange lists (Sec. 4.1,
Fig. 1): the host plan behind the sharded stage, checked on CPU against the
definitions -- own rows, ghosts = the other columns of own rows, local rows
in global order, and send/receive lists that enumerate the same values."""
import numpy as np
import pytest

from paper_2007_00094_gb300 import workloads as W

idp = pytest.importorskip("paper_2007_00094_gb300.idp")


def _pattern(mesh):
    """CSR pattern of a Q1 mesh: nodes sharing a cell are neighbours."""
    n = mesh.n_nodes
    cells = np.asarray(mesh.cells)
    k = cells.shape[1]
    a = np.repeat(cells, k, axis=1).ravel()
    b = np.tile(cells, (1, k)).ravel()
    key = np.unique(a * n + b)
    rows, cols = key // n, key % n
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    return np.cumsum(rowptr), cols.astype(np.int64)


def _meshes():
    return [W.vortex_mesh(9), W.forward_step_mesh(m=10, jitter=0.2, seed=2007),
            W.box_mesh((7, 6, 5), hi=(1.0, 1.0, 1.0), periodic=(True, False, False), jitter=0.1, seed=1),
            W.rect_mesh((9, 7), periodic=(True, False))]


def _check_plan(rowptr, col, n_shards, row_begin=None):
    n = len(rowptr) - 1
    plan = idp.ShardPlan(rowptr, col, n_shards, row_begin)
    rb = np.asarray(row_begin) if row_begin is not None else np.array([n * s // n_shards for s in range(n_shards + 1)])
    owner = np.searchsorted(rb, np.arange(n), side="right") - 1
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    local = []
    for s in range(n_shards):
        nl, lo, hi, el = plan.info(s)
        nodes = plan.nodes(s)
        own = np.arange(rb[s], rb[s + 1])
        # own rows form [lo, hi); nodes = own rows and their columns, increasing
        assert np.array_equal(nodes[lo:hi], own)
        want = np.unique(np.concatenate([own, col[rowptr[rb[s]]:rowptr[rb[s + 1]]]]))
        assert np.array_equal(nodes, want)
        lrp, lcol, entry = plan.csr(s)
        assert lrp[0] == 0 and lrp[-1] == el == len(lcol) == len(entry)
        inset = np.zeros(n, dtype=bool)
        inset[nodes] = True
        for l, g in enumerate(nodes):
            e = entry[lrp[l]:lrp[l + 1]]
            glob = np.arange(rowptr[g], rowptr[g + 1])
            # an own row keeps all its entries, a ghost row those inside the shard; same order
            keep = glob if lo <= l < hi else glob[inset[col[glob]]]
            assert np.array_equal(e, keep)
            assert np.array_equal(nodes[lcol[lrp[l]:lrp[l + 1]]], col[keep])
        local.append((nodes, lo, hi, lrp, lcol, entry))
    for s in range(n_shards):
        nodes, lo, hi, lrp, lcol, entry = local[s]
        ghosts = np.concatenate([np.arange(0, lo), np.arange(hi, len(nodes))])
        got = np.concatenate([plan.list(s, q, idp.RECV_NODES) for q in range(n_shards)] + [np.zeros(0, np.int64)])
        assert np.array_equal(np.sort(got), ghosts)  # every ghost received once
        for q in range(n_shards):
            rn = plan.list(s, q, idp.RECV_NODES)
            assert (owner[nodes[rn]] == q).all() and np.all(np.diff(nodes[rn]) > 0)
            # the sender's list and the receiver's list: the same global nodes and entries, same order
            qn = local[q][0]
            assert np.array_equal(qn[plan.list(q, s, idp.SEND_NODES)], nodes[rn])
            re = plan.list(s, q, idp.RECV_ENTRIES)
            assert np.array_equal(local[q][5][plan.list(q, s, idp.SEND_ENTRIES)], entry[re])
            # received entries: (g, i) with g a ghost owned by q and i an own row
            assert (owner[rows[entry[re]]] == q).all() and (owner[col[entry[re]]] == s).all()
        # every entry (g, i) of a ghost row into an own row is received once
        lrows = np.repeat(np.arange(len(nodes)), np.diff(lrp))
        need = np.flatnonzero(((lrows < lo) | (lrows >= hi)) & (lcol >= lo) & (lcol < hi))
        got = np.concatenate([plan.list(s, q, idp.RECV_ENTRIES) for q in range(n_shards)] + [np.zeros(0, np.int64)])
        assert np.array_equal(np.sort(got), need)
    plan.close()


@pytest.mark.parametrize("n_shards", [1, 2, 3, 5])
def test_plan_matches_definitions(n_shards):
    for mesh in _meshes():
        rowptr, col = _pattern(mesh)
        _check_plan(rowptr, col, n_shards)


def test_plan_uneven_ranges():
    rowptr, col = _pattern(W.forward_step_mesh(m=10, jitter=0.2, seed=2007))
    n = len(rowptr) - 1
    _check_plan(rowptr, col, 3, [0, 7, n // 2 + 3, n])
    _check_plan(rowptr, col, 4, [0, 1, 2, 3, n])  # shards of one row


def test_plan_rejects_bad_input():
    rowptr, col = _pattern(W.vortex_mesh(5))
    n = len(rowptr) - 1
    with pytest.raises(idp.IdpError):
        idp.ShardPlan(rowptr, col, 2, [0, 0, n])  # an empty shard
    with pytest.raises(idp.IdpError):
        idp.ShardPlan(rowptr, col, 2, [0, n // 2, n - 1])  # does not end at n
    # drop one entry (i, j) but keep (j, i): not structurally symmetric
    r0 = 3
    keep = np.ones(len(col), dtype=bool)
    k = rowptr[r0] + np.flatnonzero(col[rowptr[r0]:rowptr[r0 + 1]] != r0)[-1]
    keep[k] = False
    rp = rowptr.copy()
    rp[r0 + 1:] -= 1
    with pytest.raises(idp.IdpError):
        idp.ShardPlan(rp, col[keep], 2, [0, int(col[k]) if col[k] > r0 else r0 + 1, n])
