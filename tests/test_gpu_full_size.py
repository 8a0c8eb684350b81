"""Parity at the benchmarks' full sizes, in the launch configuration bench.py times, on sampled
blocks that the oracle computes one by one.

The device sequence is the benchmark's: the ghost regions that face a block of the same size
start as NaN on the device and cfd_exchange_ghosts fills them; cfd_autotune picks each kernel's
launch choices on these inputs; then one step (exchange + cfd_apply) as timed.  Only the
sampled blocks' outputs are read back.

- 256^3 as 512 blocks of 32^3, 4 FP64 fields (two sine sums, two Gaussian bumps of width 0.1
  domain), all 9 ops, exact tensor-core slices, n_iter 0 and 1.  Without iteration a block's
  derivatives depend on its own ghost-extended data only (mixed ops: the inner derivative on the
  rows of the outer axis's ghost zone uses the edge ghosts, Sec. "Z4c: system description").
  With one hybrid iteration (Eq. iter_center_P) a block also reads its face neighbours' closed
  solves, and for a mixed op the intermediate of those neighbours reads theirs, so the oracle
  runs on the 3 x 3 x 3 blocks around the sampled one (periodic wrap) and keeps the centre.
- The 22-field FP32 two-size layout (448 blocks of 16^3 and 64 of 32^3, coarse/fine interfaces
  with analytic ghosts) with all 9 ops on the tensor cores, n_iter 0.

Sampled blocks: corners, the blocks holding the bumps' centres (so that each field's largest
derivatives are in the sample and the relative error has the global scale), blocks on the
coarse/fine interface and seeded random ones.
"""
import numpy as np
import pytest

from oracle import cfd as C
from paper_2302_14858_gb300 import workloads as W
from tests.helpers import OPS, desc, oracle_sch, pack_fields

pytestmark = pytest.mark.gpu

TOL_EXACT64 = 1e-7
TOL_EXACT32 = 1e-6


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


def ghost_mask(N, g):
    """Flat E^3 mask of the ghost points of one block (z, y, x order)."""
    E = N + 2 * g
    m = np.ones((E, E, E), bool)
    m[g:g + N, g:g + N, g:g + N] = False
    return m.reshape(-1)


def run_bench_sequence(lib, torch, B, host_buf, nf, prec, n_iter, sample, mesh):
    """exchange -> autotune -> exchange + apply, as bench.py; the sampled blocks' outputs."""
    dev = torch.device("cuda", 0)
    fields = torch.from_numpy(host_buf).to(dev)
    nops = len(OPS)
    nint = int(sum(int(n) ** 3 for n in mesh.n))
    out = torch.full((nint * nf * nops,), float("nan"), dtype=fields.dtype, device=dev)
    ws = lib.cfd_apply_workspace(B, nf, lib.CFD_OP_ALL, prec, n_iter)
    work = torch.empty(max(ws, 256), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    lib.cfd_exchange_ghosts(B, fields, nf, stream)
    lib.cfd_autotune(B, fields, nf, lib.CFD_OP_ALL, prec, n_iter, out, work, stream)
    out.fill_(float("nan"))
    lib.cfd_exchange_ghosts(B, fields, nf, stream)
    lib.cfd_apply(B, fields, nf, lib.CFD_OP_ALL, prec, n_iter, out, work, stream)
    lib.cfd_sync_status(B, stream)
    torch.cuda.synchronize()
    offs = np.concatenate([[0], np.cumsum([int(n) ** 3 * nf * nops for n in mesh.n])])
    got = {b: out[offs[b]:offs[b + 1]].cpu().numpy().reshape(nf, nops, *(3 * [int(mesh.n[b])]))
           for b in sample}
    ext_offs = np.concatenate([[0], np.cumsum([(int(n) + 2 * mesh.g) ** 3 * nf for n in mesh.n])])
    ext = {b: fields[ext_offs[b]:ext_offs[b + 1]].cpu().numpy() for b in sample}
    del fields, out, work
    torch.cuda.empty_cache()
    return got, ext


def compare(got, want, sample, nf):
    """max over fields and ops of max |got - want| / max |want|, both maxima over the sample."""
    worst = {}
    for q in range(nf):
        for i, op in enumerate(OPS):
            den = max(np.abs(want[b][q][op]).max() for b in sample)
            err = max(np.abs(got[b][q, i].astype(np.float64) - want[b][q][op]).max() for b in sample)
            worst[(q, op)] = err / den
    return worst


@pytest.fixture(scope="module")
def cfd256():
    """256^3, 4 FP64 fields of the precision-form workload, ghosts filled by the oracle."""
    NM, N, g = 256, 32, 4
    fs = W.workload_fields(3)
    dx = 2 * np.pi / NM
    x = (np.arange(NM) + 0.5) * dx
    exts = []
    for f in fs:
        fg = np.broadcast_to(f(x[None, None, :], x[None, :, None], x[:, None, None]), (NM, NM, NM))
        exts.append(C.ghost_fill_3d(np.ascontiguousarray(fg), N, g))
    nb = NM // N
    # sample: two opposite corners, the blocks holding the two bumps' centres, three seeded others
    sample = {(0, 0, 0), (nb - 1, nb - 1, nb - 1)}
    for f in fs:
        if isinstance(f, W.PeriodicGaussian):
            cx, cy, cz = (np.floor(np.asarray(f.c) / (N * dx)).astype(int) % nb)
            sample.add((int(cz), int(cy), int(cx)))
    r = W.rng(256 + 32)
    while len(sample) < 7:
        sample.add(tuple(int(v) for v in r.integers(0, nb, size=3)))
    return NM, N, g, dx, fs, exts, sorted(sample)


@pytest.mark.parametrize("n_iter", [0, 1])
def test_default_workload_full_size_sampled_blocks(lib, torch, cfd256, n_iter):
    NM, N, g, dx, fs, exts, sample3 = cfd256
    nb, nf = NM // N, len(fs)
    mesh = W.uniform_mesh(NM, N, g)
    sample = [(bz * nb + by) * nb + bx for bz, by, bx in sample3]
    host = pack_fields(exts).reshape(mesh.nblocks, nf, -1)
    gm = ghost_mask(N, g)
    truth = {b: host[b].copy() for b in sample}
    host[:, :, gm] = np.nan            # every region has a same-size neighbour: the exchange fills all
    host = host.reshape(-1)
    s = lib.cfd_scheme_create(desc("Q13_1_d1"), desc("Q13_1_d2"))
    B = lib.cfd_blocks_bind(s, mesh.n, mesh.dx, mesh.neighbors, g, lib.CFD_F64)
    got, ext = run_bench_sequence(lib, torch, B, host, nf, lib.CFD_TC_BF16_EXACT, n_iter, sample, mesh)
    del host
    for b in sample:                   # the exchange wrote exactly the oracle's ghosts (Eq. example_G)
        assert np.array_equal(ext[b].reshape(nf, -1), truth[b]), b
    s1, s2 = oracle_sch("Q13_1_d1"), oracle_sch("Q13_1_d2")
    want = {}
    for b, (bz, by, bx) in zip(sample, sample3):
        want[b] = []
        for q in range(nf):
            if n_iter == 0:
                want[b].append(C.apply_block(exts[q][bz, by, bx], s1, s2, (dx, dx, dx), N, g, OPS))
            else:
                zs, ys, xs = ([(c + d) % nb for d in (-1, 0, 1)] for c in (bz, by, bx))
                res = C.apply_uniform(exts[q][np.ix_(zs, ys, xs)], s1, s2, (dx, dx, dx), N, g, OPS, n_iter)
                want[b].append({op: v[1, 1, 1] for op, v in res.items()})
    worst = compare(got, want, sample, nf)
    print(f"256^3/32^3 n_iter {n_iter}, {len(sample)} sampled blocks: max rel err", max(worst.values()))
    for k, v in worst.items():
        assert v < TOL_EXACT64, (k, v)


def test_two_size_fp32_workload_full_size_sampled_blocks(lib, torch):
    """448 x 16^3 + 64 x 32^3, 22 FP32 fields, 9 ops: regions facing a same-size block come from
    the exchange, those facing the other level hold analytic values (neighbour -1)."""
    mesh = W.box_in_box_mesh(4)
    g = mesh.g
    fs = W.workload_fields(4)
    nf = len(fs)
    per_block = W.sample(mesh, fs, dtype=np.float32)
    # sample: the first coarse block, coarse and fine blocks on the level interface, seeded others
    nmiss = (mesh.neighbors < 0).sum(1)
    coarse = np.flatnonzero(mesh.n == 16)
    fine = np.flatnonzero(mesh.n == 32)
    sample = {int(coarse[0]), int(coarse[np.argmax(nmiss[coarse])]), int(fine[np.argmax(nmiss[fine])]),
              int(fine[np.argmin(nmiss[fine])])}
    r = W.rng(448 + 64)
    while len(sample) < 7:
        sample.add(int(r.integers(0, mesh.nblocks)))
    sample = sorted(sample)
    # oracle ghosts: the same-size neighbours' interiors (Eq. example_G), per size group
    ref = {}
    for q in range(nf):
        blocks_q = [per_block[b][q].astype(np.float64) for b in range(mesh.nblocks)]
        for n in np.unique(mesh.n):
            nbr = mesh.neighbors.copy()
            nbr[mesh.n != n] = -1
            blocks_q = C.exchange_ghosts(blocks_q, nbr, int(n), g)
        for b in sample:
            ref.setdefault(b, []).append(blocks_q[b])
    for b in range(mesh.nblocks):
        n = int(mesh.n[b])
        for rr, (dz, dy, dxx) in enumerate(W.DIRS):
            if mesh.neighbors[b, rr] >= 0:
                part = {-1: slice(0, g), 0: slice(g, g + n), 1: slice(g + n, 2 * g + n)}
                per_block[b][:, part[dz], part[dy], part[dxx]] = np.nan
    host = W.pack(per_block)
    del per_block
    s = lib.cfd_scheme_create(desc("Q13_1_d1"), desc("Q13_1_d2"))
    B = lib.cfd_blocks_bind(s, mesh.n, mesh.dx, mesh.neighbors, g, lib.CFD_F32)
    got, ext = run_bench_sequence(lib, torch, B, host, nf, lib.CFD_TC_BF16_EXACT, 0, sample, mesh)
    for b in sample:
        E = int(mesh.n[b]) + 2 * g
        e = ext[b].reshape(nf, E, E, E).astype(np.float64)
        for q in range(nf):
            assert np.array_equal(e[q], ref[b][q]), (b, q)
    s1, s2 = oracle_sch("Q13_1_d1"), oracle_sch("Q13_1_d2")
    want = {b: [C.apply_block(ref[b][q], s1, s2, mesh.dx[b], int(mesh.n[b]), g, OPS) for q in range(nf)]
            for b in sample}
    worst = compare(got, want, sample, nf)
    print(f"two-size FP32, {len(sample)} sampled blocks: max rel err", max(worst.values()))
    for k, v in worst.items():
        assert v < TOL_EXACT32, (k, v)
