"""Domain decomposition across ranks: the partition plan of gks_partition_create (owned cells,
halo cells and send lists) and the data movement it plans, by torch.distributed point-to-point
messages (gloo on CPU tensors, NCCL on device tensors). A two-stage step exchanges the halo of
the state and of the stage state; the time step is the minimum over the ranks.

States here are [5][n_cells] arrays in the caller's cell order, of which a rank keeps its owned
and halo columns current.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import GksError, GKS_OK, load_library, Mesh


class Partition:
    """The plan of one rank: owned (Morton order), halo (by owning rank, then id), halo_owner,
    and send[q] (the owned cells that rank q reads, in q's halo order)."""

    def __init__(self, mesh: Mesh, nranks: int, rank: int):
        L = load_library()
        h = ctypes.c_void_p()
        s = L.gks_partition_create(mesh.h, int(nranks), int(rank), ctypes.byref(h))
        if s != GKS_OK:
            raise GksError(s, L.gks_last_error(None).decode())
        try:
            no, nh = ctypes.c_int64(), ctypes.c_int64()
            L.gks_partition_counts(h, ctypes.byref(no), ctypes.byref(nh))
            self.owned = np.zeros(no.value, dtype=np.int64)
            self.halo = np.zeros(nh.value, dtype=np.int64)
            self.halo_owner = np.zeros(nh.value, dtype=np.int32)
            L.gks_partition_cells(h, self.owned.ctypes.data, self.halo.ctypes.data,
                                  self.halo_owner.ctypes.data)
            self.send = []
            for q in range(nranks):
                n = ctypes.c_int64()
                L.gks_partition_send(h, q, ctypes.byref(n), None)
                cells = np.zeros(n.value, dtype=np.int64)
                L.gks_partition_send(h, q, ctypes.byref(n), cells.ctypes.data)
                self.send.append(cells)
        finally:
            L.gks_partition_destroy(h)
        self.nranks, self.rank = nranks, rank
        self.recv = [self.halo[self.halo_owner == q] for q in range(nranks)]


def halo_exchange(Q, part: Partition, dist, group=None):
    """Fill the halo columns of Q (torch tensor [5][n], caller order) from their owners: every
    rank sends the columns its peers read and receives its own halo, all messages in flight at
    once."""
    import torch
    reqs, inbox = [], []
    for q in range(part.nranks):
        if q == part.rank:
            continue
        if len(part.send[q]):
            idx = torch.from_numpy(part.send[q]).to(Q.device)
            buf = Q[:, idx].contiguous()
            reqs.append(dist.isend(buf, dst=q, group=group))
        if len(part.recv[q]):
            buf = torch.empty((Q.shape[0], len(part.recv[q])), dtype=Q.dtype, device=Q.device)
            reqs.append(dist.irecv(buf, src=q, group=group))
            inbox.append((q, buf))
    for r in reqs:
        r.wait()
    for q, buf in inbox:
        Q[:, torch.from_numpy(part.recv[q]).to(Q.device)] = buf
    return Q


def global_min_dt(dt_local: float, dist, device="cpu", group=None) -> float:
    """The step every rank takes: the minimum of the ranks' CFL bounds."""
    import torch
    t = torch.tensor([float(dt_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MIN, group=group)
    return float(t.item())
