"""Halo exchange of the sharded stage between ranks (Sec. 4.1, Fig. 1-2).

One rank holds one shard of a :class:`~paper_2007_00094_gb300.idp.ShardPlan`
(its rows and one ghost layer).  At the stage's synchronisation points it
sends the values of its rows that other shards hold as ghosts and receives
its ghosts' values: node arrays (alpha, R, U; ``exchange_nodes``) and the
limiter values of ghost rows' entries into its rows (``exchange_entries``),
plus the min-reduction of the CFL bound (``min_allreduce``).  Both sides of a
link enumerate the same values in the order of global ids (the plan's
lists), so a message is a packed array with no index attached.

This is the transport for one process per GPU over ``torch.distributed``:
it moves whatever tensors it is given (CPU tensors over gloo, device tensors
over NCCL).  Within one process, ``idp_shards_*`` runs every shard on one GPU
with the same lists and device copies instead.
"""
from __future__ import annotations

import numpy as np

from .idp import RECV_ENTRIES, RECV_NODES, SEND_ENTRIES, SEND_NODES


class HaloExchange:
    def __init__(self, plan, rank: int, group=None):
        import torch

        self.rank = int(rank)
        self.group = group
        self.peers = []
        for q in range(plan.n_shards):
            if q == self.rank:
                continue
            lists = {k: torch.from_numpy(plan.list(self.rank, q, k).astype(np.int64))
                     for k in (SEND_NODES, RECV_NODES, SEND_ENTRIES, RECV_ENTRIES)}
            if any(len(v) for v in lists.values()):
                self.peers.append((q, lists))

    def _swap(self, pairs):
        """pairs: (peer, send tensor, receive tensor) -> completes all transfers."""
        import torch.distributed as dist

        ops = []
        for q, snd, rcv in pairs:
            if snd.numel():
                ops.append(dist.P2POp(dist.isend, snd, q, group=self.group))
            if rcv.numel():
                ops.append(dist.P2POp(dist.irecv, rcv, q, group=self.group))
        if ops:
            for w in dist.batch_isend_irecv(ops):
                w.wait()

    def exchange_nodes(self, X):
        """X: (comps, n_local) tensor of this shard; its ghost columns are
        overwritten with the owners' values."""
        pairs, recv = [], []
        for q, L in self.peers:
            snd = X.index_select(1, L[SEND_NODES].to(X.device)).contiguous()
            rcv = X.new_empty((X.shape[0], len(L[RECV_NODES])))
            pairs.append((q, snd, rcv))
            recv.append((L[RECV_NODES], rcv))
        self._swap(pairs)
        for idx, rcv in recv:
            X[:, idx.to(X.device)] = rcv

    def exchange_entries(self, Y):
        """Y: (nnz_local,) tensor of per-entry values of this shard (local
        CSR order); entries of ghost rows into own rows get the owners' values."""
        pairs, recv = [], []
        for q, L in self.peers:
            snd = Y.index_select(0, L[SEND_ENTRIES].to(Y.device)).contiguous()
            rcv = Y.new_empty(len(L[RECV_ENTRIES]))
            pairs.append((q, snd, rcv))
            recv.append((L[RECV_ENTRIES], rcv))
        self._swap(pairs)
        for idx, rcv in recv:
            Y[idx.to(Y.device)] = rcv

    def min_allreduce(self, t):
        """The global CFL bound: elementwise minimum over all ranks, in place."""
        import torch.distributed as dist

        dist.all_reduce(t, op=dist.ReduceOp.MIN, group=self.group)
        return t
