"""MeshBlocks of one problem split over processes (one GPU each) and the ghost exchange between them.

Host-side plumbing only: which blocks a rank owns, the local neighbour table (-1 where the
neighbour lives on another rank), and the ordered lists of ghost regions every pair of ranks
exchanges.  The copies themselves are the library's kernels (cfd_exchange_ghosts for local
neighbours, cfd_halo_pack / cfd_halo_unpack for remote ones); the transport between ranks is
torch.distributed point-to-point (NCCL between GPUs).  This is the remote part of the
communication matrix G of Eq. example_G: one halo exchange of f per apply, no reduction.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Dict, List, Tuple

import numpy as np

from . import workloads as W


def owner_ranges(nblocks: int, world: int) -> List[Tuple[int, int]]:
    """Contiguous block ranges [lo, hi) per rank (blocks in bind order)."""
    return [(r * nblocks // world, (r + 1) * nblocks // world) for r in range(world)]


def owner_of(nblocks: int, world: int) -> np.ndarray:
    own = np.empty(nblocks, np.int32)
    for r, (lo, hi) in enumerate(owner_ranges(nblocks, world)):
        own[lo:hi] = r
    return own


@dataclass
class Shard:
    rank: int
    world: int
    blocks: np.ndarray                  # global ids owned, in local order
    mesh: W.Mesh                        # local blocks; neighbours as local ids, -1 where remote
    send: Dict[int, List[Tuple[int, int]]]   # peer -> [(local owner block, direction)]
    recv: Dict[int, List[Tuple[int, int]]]   # peer -> [(local receiving block, direction)]


def shard(mesh: W.Mesh, world: int, rank: int) -> Shard:
    """The part of ``mesh`` that ``rank`` owns and its exchange lists.

    A ghost region (receiving block B, direction r) whose neighbour NB = neighbors[B, r] is
    owned by another rank is sent by owner(NB) and received by owner(B); both sides list these
    regions sorted by (B, r), so the k-th item of a send list and of the matching receive list
    describe the same region."""
    nb = mesh.nblocks
    own = owner_of(nb, world)
    lo, hi = owner_ranges(nb, world)[rank]
    ids = np.arange(lo, hi)
    local = {int(b): i for i, b in enumerate(ids)}
    nbr = np.full((len(ids), 26), -1, np.int32)
    for i, b in enumerate(ids):
        for r in range(26):
            v = int(mesh.neighbors[b, r])
            if v >= 0 and own[v] == rank:
                nbr[i, r] = local[v]
    send: Dict[int, List[Tuple[int, int]]] = {}
    recv: Dict[int, List[Tuple[int, int]]] = {}
    for B in range(nb):
        for r in range(26):
            NB = int(mesh.neighbors[B, r])
            if NB < 0 or own[NB] == own[B]:
                continue
            if own[B] == rank:
                recv.setdefault(int(own[NB]), []).append((local[B], r))
            if own[NB] == rank:
                send.setdefault(int(own[B]), []).append((local[NB], r))
    sub = W.Mesh(mesh.n[ids], mesh.origin[ids], mesh.dx[ids], nbr, mesh.g)
    return Shard(rank, world, ids, sub, send, recv)


class ShardedExchange:
    """Ghost exchange of a rank's blocks: local neighbours by cfd_exchange_ghosts, remote ones by
    pack -> point-to-point transfer -> unpack (receives posted before sends, then waited)."""

    def __init__(self, cfd, blocks, sh: Shard, nfields: int, device, dtype):
        import torch
        self.cfd, self.blocks, self.sh, self.nf = cfd, blocks, sh, nfields
        self.pack_plans = {p: cfd.cfd_halo_plan_create(blocks, items) for p, items in sh.send.items()}
        self.unpack_plans = {p: cfd.cfd_halo_plan_create(blocks, items) for p, items in sh.recv.items()}
        esz = torch.empty((), dtype=dtype).element_size()
        self.sendbuf = {p: torch.empty(cfd.cfd_halo_plan_bytes(pl, nfields) // esz, dtype=dtype, device=device)
                        for p, pl in self.pack_plans.items()}
        self.recvbuf = {p: torch.empty(cfd.cfd_halo_plan_bytes(pl, nfields) // esz, dtype=dtype, device=device)
                        for p, pl in self.unpack_plans.items()}

    def exchange(self, fields, stream=None):
        import torch.distributed as dist
        self.cfd.cfd_exchange_ghosts(self.blocks, fields, self.nf, stream)
        for p, pl in self.pack_plans.items():
            self.cfd.cfd_halo_pack(pl, fields, self.nf, self.sendbuf[p], stream)
        reqs = [dist.irecv(buf, src=p) for p, buf in self.recvbuf.items()]
        reqs += [dist.isend(buf, dst=p) for p, buf in self.sendbuf.items()]
        for q in reqs:
            q.wait()
        for p, pl in self.unpack_plans.items():
            self.cfd.cfd_halo_unpack(pl, fields, self.nf, self.recvbuf[p], stream)
