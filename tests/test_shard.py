"""Splitting the blocks over processes: the exchange lists of paper_2302_14858_gb300/shard.py,
run on CPU with world_size 2 (gloo) and a plain-numpy copy of each listed ghost region, fill every
ghost region exactly as the single-process ghost fill does (Eq. example_G)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DIRS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1) if (dz, dy, dx) != (0, 0, 0)]


def _region(d, N, g):
    return {-1: range(-g, 0), 0: range(0, N), 1: range(N, N + g)}[d]


def np_pack(blocks, items, N, g):
    """The owner's interior slab for each (owner block, direction) item, (z, y, x) order."""
    out = []
    for b, r in items:
        dz, dy, dx = DIRS[r]
        for z in _region(dz, N, g):
            for y in _region(dy, N, g):
                for x in _region(dx, N, g):
                    out.append(blocks[b][z - dz * N + g, y - dy * N + g, x - dx * N + g])
    return np.asarray(out)


def np_unpack(blocks, items, N, g, buf):
    k = 0
    for b, r in items:
        dz, dy, dx = DIRS[r]
        for z in _region(dz, N, g):
            for y in _region(dy, N, g):
                for x in _region(dx, N, g):
                    blocks[b][z + g, y + g, x + g] = buf[k]
                    k += 1
    assert k == len(buf)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import cfd as C
        from paper_2302_14858_gb300 import shard as SH
        from paper_2302_14858_gb300 import workloads as W
        NM, N, g = 32, 8, 4
        mesh = W.uniform_mesh(NM, N, g)
        sh = SH.shard(mesh, world, rank)
        rng = np.random.default_rng(7)
        fg = rng.standard_normal((NM, NM, NM))
        ext = C.ghost_fill_3d(fg, N, g).reshape(mesh.nblocks, N + 2 * g, N + 2 * g, N + 2 * g)
        # each rank starts from its own blocks' interiors only
        mine = []
        for b in sh.blocks:
            blk = np.zeros_like(ext[b])
            blk[g:g + N, g:g + N, g:g + N] = ext[b][g:g + N, g:g + N, g:g + N]
            mine.append(blk)
        mine = C.exchange_ghosts(mine, sh.mesh.neighbors, N, g)       # local neighbours
        reqs, recv = [], {}
        for p, items in sh.recv.items():
            recv[p] = torch.empty(len(items) and sum(
                int(np.prod([N if d == 0 else g for d in DIRS[r]])) for _, r in items), dtype=torch.float64)
            reqs.append(dist.irecv(recv[p], src=p))
        for p, items in sh.send.items():
            reqs.append(dist.isend(torch.from_numpy(np_pack(mine, items, N, g)), dst=p))
        for r_ in reqs:
            r_.wait()
        for p, items in sh.recv.items():
            np_unpack(mine, items, N, g, recv[p].numpy())
        err = max(float(np.abs(mine[i] - ext[b]).max()) for i, b in enumerate(sh.blocks))
        q.put((rank, err, len(sh.blocks), {p: len(v) for p, v in sh.send.items()}))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_ranks_fill_every_ghost_region():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(240)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    res = sorted(q.get() for _ in range(world))
    for rank, err, nown, sends in res:
        assert err == 0.0                    # bit-exact copies
        assert nown == 32                    # 64 blocks split evenly
        assert sends and all(v > 0 for v in sends.values())


def test_exchange_lists_match_between_ranks():
    """For every pair of ranks the k-th sent region is the k-th received region (same receiver
    block and direction), for an uneven split over 3 ranks."""
    import sys
    sys.path.insert(0, ROOT)
    from paper_2302_14858_gb300 import shard as SH
    from paper_2302_14858_gb300 import workloads as W
    mesh = W.uniform_mesh(48, 16, 4)       # 27 blocks
    world = 3
    shards = [SH.shard(mesh, world, r) for r in range(world)]
    for s in shards:
        for p, items in s.send.items():
            mine = [(int(s.blocks[b]), r) for b, r in items]
            theirs = [(int(shards[p].blocks[b]), r) for b, r in shards[p].recv[s.rank]]
            # the sender lists (owner, r); the receiver (B, r) with neighbors[B, r] = owner
            assert [int(mesh.neighbors[B, r]) for B, r in theirs] == [o for o, _ in mine]
            assert [r for _, r in theirs] == [r for _, r in mine]
    # every remote neighbour relation appears exactly once
    total = sum(len(v) for s in shards for v in s.recv.values())
    own = SH.owner_of(mesh.nblocks, world)
    want = sum(1 for B in range(mesh.nblocks) for r in range(26) if own[mesh.neighbors[B, r]] != own[B])
    assert total == want
