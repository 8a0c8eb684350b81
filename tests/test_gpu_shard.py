"""The remote ghost exchange kernels (cfd_halo_pack / cfd_halo_unpack) with the exchange lists of
paper_2302_14858_gb300/shard.py, ranks emulated in one process on one GPU (each rank its own
bound handle and buffer; the transfer between ranks is a device copy, no kernel waits on another):
the ghost regions equal the single-process fill bit for bit, and the derivatives on the split
blocks equal the oracle's on the whole mesh."""
import numpy as np
import pytest

from oracle import cfd as C
from tests.helpers import OPS, desc, oracle_sch, rel_max

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2302_14858_gb300 import build
    build.build()
    from paper_2302_14858_gb300 import cfd
    return cfd


@pytest.fixture(scope="module")
def torch():
    import torch
    return torch


@pytest.mark.parametrize("world,dtype", [(2, np.float64), (3, np.float64), (2, np.float32)])
def test_emulated_ranks(lib, torch, world, dtype):
    from paper_2302_14858_gb300 import shard as SH
    from paper_2302_14858_gb300 import workloads as W
    NM, N, g, nf = 48, 16, 4, 2
    E = N + 2 * g
    mesh = W.uniform_mesh(NM, N, g)
    rng = np.random.default_rng(11)
    fgs = [rng.standard_normal((NM, NM, NM)) for _ in range(nf)]
    exts = [C.ghost_fill_3d(f, N, g).reshape(mesh.nblocks, E, E, E) for f in fgs]
    shards = [SH.shard(mesh, world, r) for r in range(world)]
    s = lib.cfd_scheme_create(desc("Q13_1_d1"), desc("Q13_1_d2"))
    cdt = lib.CFD_F64 if dtype == np.float64 else lib.CFD_F32
    handles, bufs = [], []
    for sh in shards:
        handles.append(lib.cfd_blocks_bind(s, sh.mesh.n, sh.mesh.dx, sh.mesh.neighbors, g, cdt))
        loc = np.zeros((len(sh.blocks), nf, E, E, E), dtype)
        for i, b in enumerate(sh.blocks):
            for q in range(nf):
                loc[i, q][g:g + N, g:g + N, g:g + N] = exts[q][b][g:g + N, g:g + N, g:g + N]
        bufs.append(torch.from_numpy(loc.reshape(-1).copy()).cuda())
    tdt = torch.float64 if dtype == np.float64 else torch.float32
    for r, sh in enumerate(shards):
        lib.cfd_exchange_ghosts(handles[r], bufs[r], nf)
    # pack on every owner, "send" by a device copy, unpack on every receiver
    plans = []
    for r, sh in enumerate(shards):
        for p, items in sh.send.items():
            pk = lib.cfd_halo_plan_create(handles[r], items)
            up = lib.cfd_halo_plan_create(handles[p], shards[p].recv[r])
            nb = lib.cfd_halo_plan_bytes(pk, nf)
            assert nb == lib.cfd_halo_plan_bytes(up, nf)
            send = torch.empty(nb // np.dtype(dtype).itemsize, dtype=tdt, device="cuda")
            lib.cfd_halo_pack(pk, bufs[r], nf, send)
            recv = send.clone()
            lib.cfd_halo_unpack(up, bufs[p], nf, recv)
            plans += [pk, up]
    torch.cuda.synchronize()
    for r, sh in enumerate(shards):
        got = bufs[r].cpu().numpy().reshape(len(sh.blocks), nf, E, E, E)
        for i, b in enumerate(sh.blocks):
            for q in range(nf):
                assert np.array_equal(got[i, q], exts[q][b].astype(dtype)), (r, i, q)
    if dtype != np.float64:
        return
    # the split blocks give the whole mesh's derivatives (closures only: the iteration needs the
    # neighbours' k^c values, which stay within a process)
    s1, s2 = oracle_sch("Q13_1_d1"), oracle_sch("Q13_1_d2")
    ref = C.apply_uniform(exts[0].reshape(3, 3, 3, E, E, E), s1, s2, (2 * np.pi / NM,) * 3, N, g, OPS, 0)
    for r, sh in enumerate(shards):
        nbk = len(sh.blocks)
        out = torch.empty(nbk * nf * 9 * N ** 3, dtype=torch.float64, device="cuda")
        ws = lib.cfd_apply_workspace(handles[r], nf, lib.CFD_OP_ALL, lib.CFD_FP64_BANDED, 0)
        work = torch.empty(max(ws, 256), dtype=torch.uint8, device="cuda")
        lib.cfd_apply(handles[r], bufs[r], nf, lib.CFD_OP_ALL, lib.CFD_FP64_BANDED, 0, out, work)
        lib.cfd_sync_status(handles[r])
        got = out.cpu().numpy().reshape(nbk, nf, 9, N, N, N)
        for i, op in enumerate(OPS):
            want = ref[op].reshape(mesh.nblocks, N, N, N)[sh.blocks]
            assert rel_max(got[:, 0, i], want) < 1e-12, (r, op)


def test_plan_rejects_bad_items(lib, torch):
    from paper_2302_14858_gb300 import workloads as W
    mesh = W.uniform_mesh(32, 16, 4)
    s = lib.cfd_scheme_create(desc("Q13_1_d1"), None)
    B = lib.cfd_blocks_bind(s, mesh.n, mesh.dx, mesh.neighbors, 4, lib.CFD_F64)
    with pytest.raises(lib.CfdError):
        lib.cfd_halo_plan_create(B, [(0, 26)])
    with pytest.raises(lib.CfdError):
        lib.cfd_halo_plan_create(B, [(8, 0)])
    empty = lib.cfd_halo_plan_create(B, np.zeros((0, 2), np.int32))
    assert lib.cfd_halo_plan_bytes(empty, 3) == 0
