"""GPU parity of the tensor-core dense path (tcgen05, BF16 digit slices) against the oracle.

Tolerances (relative max error per field and op, against the FP64 oracle):
  exact slices (CFD_TC_BF16_EXACT)  <= 1e-7 on FP64 fields: the design bound is
      ~2^-37 of sum_j |D_ij f_j| (discarded slice pairs and digit remainders),
      times the cancellation sum_j |D_ij f_j| / max |D f|.  That factor grows
      like dx^-d: ~370 for d_xx of a Gaussian at 64^3 (measured error 2.8e-9),
      ~6000 at 256^3 (one stage: 4.4e-8; a mixed op chains two stages, and
      the 256^3 workload measures 6.2e-8, test_gpu_full_size.py).  The
      contract of the path is 1e-6;
  exact slices on FP32 fields     <= 1e-6 (one FP32 rounding of the output dominates);
  3-product split (CFD_TC_BF16X3)   measured bound, asserted <= 5e-2 (not an FP64-grade mode).
"""
import numpy as np
import pytest

from oracle import cfd as C
from paper_2302_14858_gb300 import workloads as W
from tests.helpers import OPS, desc, oracle_sch, rel_max

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


def apply(lib, torch, B, buf, nf, mask, prec, n_iter=0, dtype=np.float64):
    dev = torch.device("cuda", 0)
    fields = torch.from_numpy(np.ascontiguousarray(buf.astype(dtype))).to(dev)
    nops = bin(mask).count("1")
    nint = sum(int(n) ** 3 for n in B.block_n)
    out = torch.full((nint * nf * nops,), float("nan"), dtype=fields.dtype, device=dev)
    ws = lib.cfd_apply_workspace(B, nf, mask, prec, n_iter)
    work = torch.empty(max(ws, 256), dtype=torch.uint8, device=dev)
    lib.cfd_apply(B, fields, nf, mask, prec, n_iter, out, work)
    lib.cfd_sync_status(B)
    return out.cpu().numpy()


def uniform(NM, N, g, fields):
    mesh = W.uniform_mesh(NM, N, g)
    dx = 2 * np.pi / NM
    x = (np.arange(NM) + 0.5) * dx
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    exts = [C.ghost_fill_3d(f(X, Y, Z), N, g) for f in fields]
    E = N + 2 * g
    buf = np.stack([e.reshape(mesh.nblocks, E, E, E) for e in exts], axis=1).reshape(-1)
    return mesh, dx, exts, buf


def fields4(seed):
    r = W.rng(seed)
    return [W.sine_sum(r, 8, 1, 12), W.gaussian(r, 0.1), W.sine_sum(r, 8, 1, 12), W.gaussian(r, 0.1)]


@pytest.mark.parametrize("NM,N", [(64, 16), (64, 32), (128, 32)])
def test_exact_slices_all_ops(lib, torch, NM, N):
    g = 4
    fs = fields4(300 + NM + N)
    mesh, dx, exts, buf = uniform(NM, N, g, fs)
    s = lib.cfd_scheme_create(desc("Q13_1_d1"), desc("Q13_1_d2"))
    B = lib.cfd_blocks_bind(s, mesh.n, mesh.dx, mesh.neighbors, g, lib.CFD_F64)
    nf = len(fs)
    got = apply(lib, torch, B, buf, nf, lib.CFD_OP_ALL, lib.CFD_TC_BF16_EXACT).reshape(mesh.nblocks, nf, 9, N, N, N)
    s1, s2 = oracle_sch("Q13_1_d1"), oracle_sch("Q13_1_d2")
    worst = {}
    for q in range(nf):
        ref = C.apply_uniform(exts[q], s1, s2, (dx, dx, dx), N, g, OPS, 0)
        for i, op in enumerate(OPS):
            worst[(q, op)] = rel_max(got[:, q, i], ref[op].reshape(mesh.nblocks, N, N, N))
    print("exact-slice max rel err", max(worst.values()))
    for k, v in worst.items():
        assert v < TOL_EXACT64, (k, v)


@pytest.mark.parametrize("NM,N,n_iter,nf", [(64, 16, 1, 4), (64, 16, 2, 2), (64, 32, 1, 2), (128, 32, 2, 1)])
def test_exact_slices_hybrid_iteration(lib, torch, NM, N, n_iter, nf):
    """Eq. iter_center_P on the tensor cores: halo passes + iterated operator vs the oracle."""
    g = 4
    r = W.rng(500 + NM + N + n_iter)
    fs = [W.sine_sum(r, 8, 1, 12) for _ in range(nf)]  # non-zero on every block face
    mesh, dx, exts, buf = uniform(NM, N, g, fs)
    s = lib.cfd_scheme_create(desc("Q13_1_d1"), desc("Q13_1_d2"))
    B = lib.cfd_blocks_bind(s, mesh.n, mesh.dx, mesh.neighbors, g, lib.CFD_F64)
    got = apply(lib, torch, B, buf, nf, lib.CFD_OP_ALL, lib.CFD_TC_BF16_EXACT, n_iter).reshape(
        mesh.nblocks, nf, 9, N, N, N)
    s1, s2 = oracle_sch("Q13_1_d1"), oracle_sch("Q13_1_d2")
    worst = {}
    for q in range(nf):
        ref = C.apply_uniform(exts[q], s1, s2, (dx, dx, dx), N, g, OPS, n_iter)
        closed = C.apply_uniform(exts[q], s1, s2, (dx, dx, dx), N, g, OPS, 0)
        for i, op in enumerate(OPS):
            worst[(q, op)] = rel_max(got[:, q, i], ref[op].reshape(mesh.nblocks, N, N, N))
        # the iteration moves the result far beyond the tolerance, so the comparison can tell
        assert max(rel_max(closed[op], ref[op]) for op in OPS) > 10 * TOL_EXACT64
    print("iterated exact-slice max rel err", max(worst.values()))
    for k, v in worst.items():
        assert v < TOL_EXACT64, (k, v)


def test_exact_slices_iteration_matches_banded_full_size(lib, torch):
    """128^3 as 512 blocks of 16^3, one hybrid iteration: tensor cores vs the FP64 banded solve."""
    NM, N, g = 128, 16, 4
    fs = fields4(2302 + 5)
    mesh, dx, exts, buf = uniform(NM, N, g, fs)
    s = lib.cfd_scheme_create(desc("Q13_1_d1"), desc("Q13_1_d2"))
    B = lib.cfd_blocks_bind(s, mesh.n, mesh.dx, mesh.neighbors, g, lib.CFD_F64)
    tc = apply(lib, torch, B, buf, 4, lib.CFD_OP_ALL, lib.CFD_TC_BF16_EXACT, 1).reshape(mesh.nblocks, 4, 9, -1)
    fp = apply(lib, torch, B, buf, 4, lib.CFD_OP_ALL, lib.CFD_FP64_BANDED, 1).reshape(mesh.nblocks, 4, 9, -1)
    errs = [rel_max(tc[:, q, i], fp[:, q, i]) for q in range(4) for i in range(9)]
    print("iterated tc vs fp64 banded max rel err", max(errs))
    assert max(errs) < TOL_EXACT64


def test_exact_slices_iteration_periodic_block_is_cyclic(lib, torch):
    """A single periodic block has no decomposed axis: n_iter leaves the cyclic result unchanged."""
    NM = N = 16
    g = 4
    fs = fields4(91)[:1]
    mesh, dx, exts, buf = uniform(NM, N, g, fs)
    s = lib.cfd_scheme_create(desc("Q13_1_d1"), desc("Q13_1_d2"))
    B = lib.cfd_blocks_bind(s, mesh.n, mesh.dx, mesh.neighbors, g, lib.CFD_F64)
    a = apply(lib, torch, B, buf, 1, lib.CFD_OP_ALL, lib.CFD_TC_BF16_EXACT, 0)
    b = apply(lib, torch, B, buf, 1, lib.CFD_OP_ALL, lib.CFD_TC_BF16_EXACT, 2)
    assert np.array_equal(a, b)


def test_exact_slices_match_banded_fp64_full_size(lib, torch):
    """128^3 as 512 blocks of 16^3, 4 fields, 9 ops: tensor-core vs the GPU FP64 banded solve."""
    NM, N, g = 128, 16, 4
    fs = fields4(2302 + 2)
    mesh, dx, exts, buf = uniform(NM, N, g, fs)
    s = lib.cfd_scheme_create(desc("Q13_1_d1"), desc("Q13_1_d2"))
    B = lib.cfd_blocks_bind(s, mesh.n, mesh.dx, mesh.neighbors, g, lib.CFD_F64)
    tc = apply(lib, torch, B, buf, 4, lib.CFD_OP_ALL, lib.CFD_TC_BF16_EXACT).reshape(mesh.nblocks, 4, 9, -1)
    fp = apply(lib, torch, B, buf, 4, lib.CFD_OP_ALL, lib.CFD_FP64_BANDED).reshape(mesh.nblocks, 4, 9, -1)
    errs = [rel_max(tc[:, q, i], fp[:, q, i]) for q in range(4) for i in range(9)]
    print("tc vs fp64 banded max rel err", max(errs))
    assert max(errs) < TOL_EXACT64


def test_bf16x3_measured_bound(lib, torch):
    NM, N, g = 64, 16, 4
    fs = fields4(77)
    mesh, dx, exts, buf = uniform(NM, N, g, fs)
    s = lib.cfd_scheme_create(desc("Q13_1_d1"), desc("Q13_1_d2"))
    B = lib.cfd_blocks_bind(s, mesh.n, mesh.dx, mesh.neighbors, g, lib.CFD_F64)
    got = apply(lib, torch, B, buf, 4, lib.CFD_OP_ALL, lib.CFD_TC_BF16X3).reshape(mesh.nblocks, 4, 9, N, N, N)
    s1, s2 = oracle_sch("Q13_1_d1"), oracle_sch("Q13_1_d2")
    worst = 0.0
    for q in range(4):
        ref = C.apply_uniform(exts[q], s1, s2, (dx, dx, dx), N, g, OPS, 0)
        for i, op in enumerate(OPS):
            worst = max(worst, rel_max(got[:, q, i], ref[op].reshape(mesh.nblocks, N, N, N)))
    print("bf16x3 max rel err", worst)
    assert worst < 5e-2


def test_exact_slices_single_periodic_block(lib, torch):
    NM = N = 32
    g = 4
    f = W.workload_fields(1)[0]
    mesh, dx, exts, buf = uniform(NM, N, g, [f])
    s = lib.cfd_scheme_create(desc("P2_d1"), desc("P2_d2"))
    B = lib.cfd_blocks_bind(s, mesh.n, mesh.dx, mesh.neighbors, g, lib.CFD_F64)
    got = apply(lib, torch, B, buf, 1, lib.op_mask(["dx", "dyy"]), lib.CFD_TC_BF16_EXACT).reshape(2, N, N, N)
    x = (np.arange(NM) + 0.5) * dx
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    fg = f(X, Y, Z)
    want_dx = C.global_periodic(np.moveaxis(fg, 2, 0), oracle_sch("P2_d1"), dx)
    want_dyy = C.global_periodic(np.moveaxis(fg, 1, 0), oracle_sch("P2_d2"), dx)
    assert rel_max(got[0], np.moveaxis(want_dx, 0, 2)) < TOL_EXACT64
    assert rel_max(got[1], np.moveaxis(want_dyy, 0, 1)) < TOL_EXACT64


# Measured bounds of the one-product TF32 form (max relative error per op against the oracle,
# seeded sine/Gaussian fields), asserted with a factor ~2 of slack: (first-degree, second-degree,
# mixed).  Measured on GB300: 64^3 8.2e-3 / 9.3e-2 / 1.05e-1 (16^3 blocks), 7.6e-3 / 9.4e-2 /
# 1.03e-1 (32^3 blocks); 128^3 1.9e-2 / 3.7e-1 / 4.9e-1.  RMS errors are ~30x smaller.
TF32_BOUNDS = {(64, 16): (1.6e-2, 1.9e-1, 2.1e-1), (64, 32): (1.6e-2, 1.9e-1, 2.1e-1), (128, 32): (4e-2, 7.5e-1, 1.0)}


@pytest.mark.parametrize("NM,N", [(64, 16), (64, 32), (128, 32)])
def test_tf32_one_product_measured_bound(lib, torch, NM, N):
    """CFD_TC_TF32: one TF32 product with FP32 accumulation.  Its error is the TF32 rounding of
    the pencil (relative to its scale) and of D, ~2^-11 of sum_j |D_ij f_j|, times the
    cancellation sum_j |D_ij f_j| / |D f| that grows like dx^-d: a usable bound for first
    derivatives on coarse grids only.  The max and RMS relative error per op are printed and
    the measured bound is asserted per degree."""
    g = 4
    fs = fields4(700 + NM + N)
    mesh, dx, exts, buf = uniform(NM, N, g, fs)
    s = lib.cfd_scheme_create(desc("Q13_1_d1"), desc("Q13_1_d2"))
    B = lib.cfd_blocks_bind(s, mesh.n, mesh.dx, mesh.neighbors, g, lib.CFD_F64)
    nf = len(fs)
    got = apply(lib, torch, B, buf, nf, lib.CFD_OP_ALL, lib.CFD_TC_TF32).reshape(mesh.nblocks, nf, 9, N, N, N)
    s1, s2 = oracle_sch("Q13_1_d1"), oracle_sch("Q13_1_d2")
    worst = {op: 0.0 for op in OPS}
    rms = {op: 0.0 for op in OPS}
    for q in range(nf):
        ref = C.apply_uniform(exts[q], s1, s2, (dx, dx, dx), N, g, OPS, 0)
        for i, op in enumerate(OPS):
            want = ref[op].reshape(mesh.nblocks, N, N, N)
            den = np.abs(want).max()
            worst[op] = max(worst[op], rel_max(got[:, q, i], want))
            rms[op] = max(rms[op], float(np.sqrt(np.mean((got[:, q, i] - want) ** 2))) / den)
    print(f"TF32 {NM}^3/{N}^3 max rel err", {k: f"{v:.2e}" for k, v in worst.items()})
    print(f"TF32 {NM}^3/{N}^3 rms rel err", {k: f"{v:.2e}" for k, v in rms.items()})
    b1, b2, bm = TF32_BOUNDS[(NM, N)]
    for op in OPS:
        bound = b2 if op in ("dxx", "dyy", "dzz") else (bm if op in ("dxy", "dxz", "dyz") else b1)
        assert worst[op] < bound, (op, worst[op])


@pytest.mark.parametrize("n_iter", [0, 1])
def test_autotune_keeps_results_and_reports(lib, torch, n_iter):
    """cfd_autotune runs the request once with every kernel under each candidate configuration
    (TMA or cp.async staging, interleaved or contiguous tiles): the outputs are bit-identical to
    cfd_apply's, every tensor-core kernel of the request (the six stage GEMMs; the halo passes of
    the iteration run on the CUDA cores and have no choices) has a choice with its measured times,
    and cfd_apply with the tuned choices gives the same outputs again."""
    NM, N, g, nf = 64, 32, 4, 2
    mesh, dx, exts, buf = uniform(NM, N, g, fields4(811)[:nf])
    s = lib.cfd_scheme_create(desc("Q13_1_d1"), desc("Q13_1_d2"))
    B = lib.cfd_blocks_bind(s, mesh.n, mesh.dx, mesh.neighbors, g, lib.CFD_F64)
    prec = lib.CFD_TC_BF16_EXACT
    ref = apply(lib, torch, B, buf, nf, lib.CFD_OP_ALL, prec, n_iter)
    dev = torch.device("cuda", 0)
    fields = torch.from_numpy(np.ascontiguousarray(buf)).to(dev)
    out = torch.full((ref.size,), float("nan"), dtype=torch.float64, device=dev)
    ws = lib.cfd_apply_workspace(B, nf, lib.CFD_OP_ALL, prec, n_iter)
    work = torch.empty(max(ws, 256), dtype=torch.uint8, device=dev)
    lib.cfd_autotune(B, fields, nf, lib.CFD_OP_ALL, prec, n_iter, out, work)
    lib.cfd_sync_status(B)
    assert np.array_equal(out.cpu().numpy(), ref)
    rep = lib.cfd_autotune_report(B)
    (key,) = [k for k in rep if k.startswith("apply") and f"n_iter={n_iter}" in k]
    stages = rep[key]
    assert len(stages) == 6
    for st in stages:
        assert st["staging"] in ("tma", "cp.async") and st["order"] in ("interleaved", "contiguous")
        chosen = st["ms"][f"{st['staging']}/{st['order']}"]
        assert chosen > 0 and all(v < 0 or v >= chosen for v in st["ms"].values())
    again = apply(lib, torch, B, buf, nf, lib.CFD_OP_ALL, prec, n_iter)
    assert np.array_equal(again, ref)


def box16_32():
    """16^3 coarse blocks with a 2:1 refined octant of 32^3 blocks on [0, 2pi)^3 (both sizes run on
    the tensor cores): the two-size layout of the 22-field workload, 56 + 8 blocks."""
    nc = 4
    ns, origins, ds, ci, fi = [], [], [], {}, {}
    for bz in range(nc):
        for by in range(nc):
            for bx in range(nc):
                if bx < 2 and by < 2 and bz < 2:
                    continue
                ci[(bz, by, bx)] = len(ns)
                ns.append(16)
                origins.append((bx * 16, by * 16, bz * 16))
                ds.append(2 * np.pi / 64)
    for bz in range(2):
        for by in range(2):
            for bx in range(2):
                fi[(bz, by, bx)] = len(ns)
                ns.append(32)
                origins.append((bx * 32, by * 32, bz * 32))
                ds.append(np.pi / 64)
    nbr = np.full((len(ns), 26), -1, np.int32)
    for (bz, by, bx), b in ci.items():
        for r, (dz, dy, dxx) in enumerate(W.DIRS):
            nbr[b, r] = ci.get(((bz + dz) % nc, (by + dy) % nc, (bx + dxx) % nc), -1)
    for (bz, by, bx), b in fi.items():
        for r, (dz, dy, dxx) in enumerate(W.DIRS):
            nbr[b, r] = fi.get((bz + dz, by + dy, bx + dxx), -1)
    return W.Mesh(np.asarray(ns), np.asarray(origins), np.repeat(np.asarray(ds)[:, None], 3, 1), nbr, 4)


def test_exact_slices_fp32_uneven_blocks(lib, torch):
    """Blocks of 16^3 and 32^3 with analytic ghosts on the level interface, FP32 fields."""
    mesh = box16_32()
    fields = W.workload_fields(4)[:2]
    per_block = W.sample(mesh, fields, dtype=np.float32)
    buf = W.pack(per_block)
    s = lib.cfd_scheme_create(desc("Q13_1_d1"), desc("Q13_1_d2"))
    B = lib.cfd_blocks_bind(s, mesh.n, mesh.dx, mesh.neighbors, 4, lib.CFD_F32)
    out = apply(lib, torch, B, buf, 2, lib.CFD_OP_ALL, lib.CFD_TC_BF16_EXACT, dtype=np.float32)
    got = W.unpack(out, mesh, 2, interior=True, nops=9)
    s1, s2 = oracle_sch("Q13_1_d1"), oracle_sch("Q13_1_d2")
    worst = 0.0
    for q in range(2):
        for i, op in enumerate(OPS):
            want = [C.apply_block(per_block[b][q].astype(np.float64), s1, s2, mesh.dx[b], int(mesh.n[b]), 4, (op,))[op]
                    for b in range(mesh.nblocks)]
            wmax = max(np.abs(w).max() for w in want)
            err = max(np.abs(got[b][q, i].astype(np.float64) - want[b]).max() for b in range(mesh.nblocks)) / wmax
            worst = max(worst, err)
    print("fp32 exact-slice max rel err", worst)
    assert worst < TOL_EXACT32


def _ghost_slices(dz, dy, dxx, N, g):
    part = {-1: slice(0, g), 0: slice(g, g + N), 1: slice(g + N, 2 * g + N)}
    return part[dz], part[dy], part[dxx]


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_exchange_analytic_interfaces_then_apply(lib, torch, dtype):
    """The two-size workload as the benchmark runs it: cfd_exchange_ghosts fills every region
    that faces a block of the same size (those regions start as NaN on the device), the
    regions facing the other level hold analytic values (neighbour -1), then all 9 ops on
    the tensor cores.  Oracle: the same exchange in numpy (Eq. example_G) per size group,
    then the closed block operators per block."""
    mesh = box16_32()
    g, nf = 4, 2
    fields = W.workload_fields(4)[:nf]
    per_block = W.sample(mesh, fields, dtype=dtype)
    dev_blocks = [b.copy() for b in per_block]
    for b in range(mesh.nblocks):
        for r, (dz, dy, dxx) in enumerate(W.DIRS):
            if mesh.neighbors[b, r] >= 0:
                sz, sy, sx = _ghost_slices(dz, dy, dxx, int(mesh.n[b]), g)
                dev_blocks[b][:, sz, sy, sx] = np.nan
    # oracle ghosts: copies of the neighbours' interiors where a neighbour exists
    ref_blocks = []
    for q in range(nf):
        blocks_q = [per_block[b][q].astype(np.float64) for b in range(mesh.nblocks)]
        for n in np.unique(mesh.n):
            nbr = mesh.neighbors.copy()
            nbr[mesh.n != n] = -1
            blocks_q = C.exchange_ghosts(blocks_q, nbr, int(n), g)
        ref_blocks.append(blocks_q)
    s = lib.cfd_scheme_create(desc("Q13_1_d1"), desc("Q13_1_d2"))
    B = lib.cfd_blocks_bind(s, mesh.n, mesh.dx, mesh.neighbors, g,
                            lib.CFD_F32 if dtype == np.float32 else lib.CFD_F64)
    dev = torch.device("cuda", 0)
    fields_t = torch.from_numpy(W.pack(dev_blocks)).to(dev)
    lib.cfd_exchange_ghosts(B, fields_t, nf)
    nint = sum(int(n) ** 3 for n in mesh.n)
    out = torch.full((nint * nf * 9,), float("nan"), dtype=fields_t.dtype, device=dev)
    ws = lib.cfd_apply_workspace(B, nf, lib.CFD_OP_ALL, lib.CFD_TC_BF16_EXACT, 0)
    work = torch.empty(max(ws, 256), dtype=torch.uint8, device=dev)
    lib.cfd_apply(B, fields_t, nf, lib.CFD_OP_ALL, lib.CFD_TC_BF16_EXACT, 0, out, work)
    lib.cfd_sync_status(B)
    # the exchange filled exactly the oracle's ghosts
    ext = W.unpack(fields_t.cpu().numpy(), mesh, nf)
    for b in range(mesh.nblocks):
        for q in range(nf):
            assert np.array_equal(ext[b][q].astype(np.float64), ref_blocks[q][b]), (b, q)
    got = W.unpack(out.cpu().numpy(), mesh, nf, interior=True, nops=9)
    s1, s2 = oracle_sch("Q13_1_d1"), oracle_sch("Q13_1_d2")
    worst = 0.0
    for q in range(nf):
        want = [C.apply_block(ref_blocks[q][b], s1, s2, mesh.dx[b], int(mesh.n[b]), g, OPS) for b in range(mesh.nblocks)]
        for i, op in enumerate(OPS):
            wmax = max(np.abs(w[op]).max() for w in want)
            err = max(np.abs(got[b][q, i].astype(np.float64) - want[b][op]).max() for b in range(mesh.nblocks)) / wmax
            worst = max(worst, err)
    print("exchange + analytic interfaces + tensor cores, max rel err", worst)
    assert worst < (TOL_EXACT32 if dtype == np.float32 else TOL_EXACT64)


@pytest.mark.parametrize("n_iter", [0, 1])
def test_wave_rk4_tensor_cores(lib, torch, n_iter):
    """The RK4 wave driver with the tensor-core Laplacian vs the oracle's RK4 (3 steps, 64^3, 16^3 blocks)."""
    NM, N, g = 64, 16, 4
    pw = W.plane_waves(13, 4, 10.0)
    dx = 2 * np.pi / NM
    x = (np.arange(NM) + 0.5) * dx
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    phi0, K0 = pw.phi_at(0.0, X, Y, Z), pw.K_at(0.0, X, Y, Z)
    mesh = W.uniform_mesh(NM, N, g)
    s = lib.cfd_scheme_create(desc("Q13_1_d1"), desc("Q13_1_d2"))
    B = lib.cfd_blocks_bind(s, mesh.n, mesh.dx, mesh.neighbors, g, lib.CFD_F64)
    E = N + 2 * g
    pe = C.ghost_fill_3d(phi0, N, g).reshape(mesh.nblocks, E, E, E)
    ke = C.ghost_fill_3d(K0, N, g).reshape(mesh.nblocks, E, E, E)
    tp = torch.from_numpy(pe.reshape(-1).copy()).cuda()
    tk = torch.from_numpy(ke.reshape(-1).copy()).cuda()
    ws = lib.cfd_wave_workspace(B, lib.CFD_TC_BF16_EXACT, n_iter)
    work = torch.empty(ws, dtype=torch.uint8, device="cuda")
    dt = 0.25 * dx
    s2 = oracle_sch("Q13_1_d2")
    p, k = phi0, K0
    for _ in range(3):
        lib.cfd_wave_rk_step(B, tp, tk, dt, lib.CFD_TC_BF16_EXACT, n_iter, work)
        p, k = C.wave_rk4_step(p, k, dt, s2, (dx, dx, dx), N, g, n_iter)
    lib.cfd_sync_status(B)
    nb = NM // N
    gp = tp.cpu().numpy().reshape(mesh.nblocks, E, E, E)[:, g:g + N, g:g + N, g:g + N]
    gk = tk.cpu().numpy().reshape(mesh.nblocks, E, E, E)[:, g:g + N, g:g + N, g:g + N]
    gp = C.blocks_to_global(gp.reshape(nb, nb, nb, N, N, N))
    gk = C.blocks_to_global(gk.reshape(nb, nb, nb, N, N, N))
    print("wave tc rel err", rel_max(gp, p), rel_max(gk, k))
    assert rel_max(gp, p) < TOL_EXACT64
    assert rel_max(gk, k) < TOL_EXACT64


def test_cuda_graph_capture_replays_exchange_and_apply(lib, torch):
    """Ghost exchange + tensor-core apply captured in a CUDA graph: replay equals the eager result."""
    NM, N, g = 64, 16, 4
    fs = fields4(404)
    mesh, dx, exts, buf = uniform(NM, N, g, fs)
    s = lib.cfd_scheme_create(desc("Q13_1_d1"), desc("Q13_1_d2"))
    B = lib.cfd_blocks_bind(s, mesh.n, mesh.dx, mesh.neighbors, g, lib.CFD_F64)
    dev = torch.device("cuda", 0)
    fields = torch.from_numpy(buf.copy()).to(dev)
    nint = mesh.nblocks * N ** 3
    out = torch.zeros(nint * 4 * 9, dtype=torch.float64, device=dev)
    ws = lib.cfd_apply_workspace(B, 4, lib.CFD_OP_ALL, lib.CFD_TC_BF16_EXACT, 1)
    work = torch.empty(max(ws, 256), dtype=torch.uint8, device=dev)

    def step():
        lib.cfd_exchange_ghosts(B, fields, 4)
        lib.cfd_apply(B, fields, 4, lib.CFD_OP_ALL, lib.CFD_TC_BF16_EXACT, 1, out, work)

    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        step()   # eager (also sets the kernels' shared-memory opt-in before capture)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    eager = out.clone()
    out.zero_()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    graph.replay()
    graph.replay()
    torch.cuda.synchronize()
    lib.cfd_sync_status(B)
    assert torch.equal(out, eager)


@pytest.mark.parametrize("fam,n_iter", [("P1", 0), ("P2", 1), ("P3", 0), ("P3", 1)])
def test_pade_family_both_paths(lib, torch, fam, n_iter):
    """Padé P^1_{1,2,3} (4th, 6th, 8th order) with their closures P-bar_{3,4,5}: stencil widths
    M = 1..3, closure half-widths 3..5 (8th order needs 5 ghost layers), on both GPU paths."""
    NM, N = 64, 16
    g = 5 if fam == "P3" else 4
    r = W.rng(600 + int(fam[1]) + 10 * n_iter)
    fs = [W.sine_sum(r, 8, 1, 12), W.gaussian(r, 0.1)]
    mesh, dx, exts, buf = uniform(NM, N, g, fs)
    s = lib.cfd_scheme_create(desc(f"{fam}_d1"), desc(f"{fam}_d2"))
    B = lib.cfd_blocks_bind(s, mesh.n, mesh.dx, mesh.neighbors, g, lib.CFD_F64)
    s1, s2 = oracle_sch(f"{fam}_d1"), oracle_sch(f"{fam}_d2")
    tc = apply(lib, torch, B, buf, 2, lib.CFD_OP_ALL, lib.CFD_TC_BF16_EXACT, n_iter).reshape(mesh.nblocks, 2, 9, N, N, N)
    fp = apply(lib, torch, B, buf, 2, lib.CFD_OP_ALL, lib.CFD_FP64_BANDED, n_iter).reshape(mesh.nblocks, 2, 9, N, N, N)
    for q in range(2):
        ref = C.apply_uniform(exts[q], s1, s2, (dx, dx, dx), N, g, OPS, n_iter)
        for i, op in enumerate(OPS):
            want = ref[op].reshape(mesh.nblocks, N, N, N)
            assert rel_max(fp[:, q, i], want) < 1e-12, (fam, q, op)
            assert rel_max(tc[:, q, i], want) < TOL_EXACT64, (fam, q, op)


@pytest.mark.parametrize("prec,NM,N,n_iter", [(0, 32, 8, 0), (0, 32, 8, 1), (2, 64, 16, 0), (2, 64, 16, 1)])
def test_wave_lsrk_with_ko_dissipation(lib, torch, prec, NM, N, n_iter):
    """2S low-storage RK with Kreiss-Oliger dissipation (r = 4, sigma = 0.04) vs the oracle, 3 steps."""
    from oracle import timestep as T
    g, sigma, r = 4, 0.04, 4
    pw = W.plane_waves(17, 4, 10.0)
    dx = 2 * np.pi / NM
    x = (np.arange(NM) + 0.5) * dx
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    # a short-wavelength part makes the dissipation visible
    phi0 = pw.phi_at(0.0, X, Y, Z) + 0.05 * np.cos(11 * X - 9 * Y + 7 * Z)
    K0 = pw.K_at(0.0, X, Y, Z)
    mesh = W.uniform_mesh(NM, N, g)
    s = lib.cfd_scheme_create(desc("Q13_1_d1"), desc("Q13_1_d2"))
    B = lib.cfd_blocks_bind(s, mesh.n, mesh.dx, mesh.neighbors, g, lib.CFD_F64)
    E = N + 2 * g
    tp = torch.from_numpy(C.ghost_fill_3d(phi0, N, g).reshape(-1).copy()).cuda()
    tk = torch.from_numpy(C.ghost_fill_3d(K0, N, g).reshape(-1).copy()).cuda()
    work = torch.empty(lib.cfd_wave_lsrk_workspace(B, prec, n_iter), dtype=torch.uint8, device="cuda")
    coef = T.lsrk2s_rk4_float()
    dt = 0.25 * dx
    s2 = oracle_sch("Q13_1_d2")
    p, k = phi0, K0
    for _ in range(3):
        lib.cfd_wave_lsrk_step(B, tp, tk, dt, coef, sigma, r, prec, n_iter, work)
        p, k = T.wave_lsrk_step(p, k, dt, coef, s2, (dx, dx, dx), N, g, n_iter, sigma, r)
    lib.cfd_sync_status(B)
    nb = NM // N
    gp = tp.cpu().numpy().reshape(mesh.nblocks, E, E, E)[:, g:g + N, g:g + N, g:g + N]
    gk = tk.cpu().numpy().reshape(mesh.nblocks, E, E, E)[:, g:g + N, g:g + N, g:g + N]
    gp = C.blocks_to_global(gp.reshape(nb, nb, nb, N, N, N))
    gk = C.blocks_to_global(gk.reshape(nb, nb, nb, N, N, N))
    tol = 1e-12 if prec == 0 else TOL_EXACT64
    print("lsrk+ko rel err", rel_max(gp, p), rel_max(gk, k))
    assert rel_max(gp, p) < tol
    assert rel_max(gk, k) < tol
    # without dissipation the oracle's result differs well beyond the tolerance
    p0, _ = T.wave_lsrk_step(phi0, K0, dt, coef, s2, (dx, dx, dx), N, g, n_iter, 0.0, r)
    p1, _ = T.wave_lsrk_step(phi0, K0, dt, coef, s2, (dx, dx, dx), N, g, n_iter, sigma, r)
    assert rel_max(p0, p1) > 10 * tol


def test_wave_lsrk_rejects_bad_arguments(lib, torch):
    NM, N, g = 32, 16, 4
    mesh = W.uniform_mesh(NM, N, g)
    s = lib.cfd_scheme_create(desc("Q13_1_d1"), desc("Q13_1_d2"))
    B = lib.cfd_blocks_bind(s, mesh.n, mesh.dx, mesh.neighbors, g, lib.CFD_F64)
    E = N + 2 * g
    t = torch.zeros(mesh.nblocks * E ** 3, dtype=torch.float64, device="cuda")
    work = torch.empty(lib.cfd_wave_lsrk_workspace(B, 0, 0), dtype=torch.uint8, device="cuda")
    good = ([0.0, 0.5], [1.0, 0.5], [0.5, 1.0], [1.0, 1.0])
    for sigma, r in [(-0.1, 4), (0.04, 0), (0.04, 5)]:
        with pytest.raises(lib.CfdError) as e:
            lib.cfd_wave_lsrk_step(B, t, t.clone(), 0.01, good, sigma, r, 0, 0, work)
        assert e.value.status == lib.CFD_ERR_ARG
    with pytest.raises(ValueError):
        lib.cfd_wave_lsrk_step(B, t, t.clone(), 0.01, ([0.0], [1.0, 0.5], [0.5], [1.0]), 0.0, 4, 0, 0, work)


@pytest.mark.parametrize("prec", [0, 2])
def test_many_iterations_reach_the_global_scheme(lib, torch, prec):
    """Eq. iter_center_P iterated to convergence: the decomposed result becomes the undecomposed
    periodic (global) scheme, on both GPU paths (d_x and d_yy of a sine field, 8^3 blocks of 16^3)."""
    NM, N, g, n_iter = 128, 16, 4, 14
    r = W.rng(808)
    f = W.sine_sum(r, 8, 1, 12)
    mesh, dx, exts, buf = uniform(NM, N, g, [f])
    s = lib.cfd_scheme_create(desc("Q13_1_d1"), desc("Q13_1_d2"))
    B = lib.cfd_blocks_bind(s, mesh.n, mesh.dx, mesh.neighbors, g, lib.CFD_F64)
    got = apply(lib, torch, B, buf, 1, lib.op_mask(["dx", "dyy"]), prec, n_iter).reshape(mesh.nblocks, 2, N, N, N)
    x = (np.arange(NM) + 0.5) * dx
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    fg = f(X, Y, Z)
    want_dx = np.moveaxis(C.global_periodic(np.moveaxis(fg, 2, 0), oracle_sch("Q13_1_d1"), dx), 0, 2)
    want_dyy = np.moveaxis(C.global_periodic(np.moveaxis(fg, 1, 0), oracle_sch("Q13_1_d2"), dx), 0, 1)
    nb = NM // N
    gdx = C.blocks_to_global(got[:, 0].reshape(nb, nb, nb, N, N, N))
    gdyy = C.blocks_to_global(got[:, 1].reshape(nb, nb, nb, N, N, N))
    tol = 1e-10 if prec == 0 else TOL_EXACT64
    print("iterated to the global scheme", rel_max(gdx, want_dx), rel_max(gdyy, want_dyy))
    assert rel_max(gdx, want_dx) < tol
    assert rel_max(gdyy, want_dyy) < tol


def test_tensor_cores_reject_unsupported_block_size(lib, torch):
    """The dense operators are built for N = 16 and 32 only: N = 8 blocks are refused, not computed."""
    NM, N, g = 32, 8, 4
    mesh = W.uniform_mesh(NM, N, g)
    s = lib.cfd_scheme_create(desc("Q13_1_d1"), desc("Q13_1_d2"))
    B = lib.cfd_blocks_bind(s, mesh.n, mesh.dx, mesh.neighbors, g, lib.CFD_F64)
    buf = np.zeros(mesh.nblocks * (N + 2 * g) ** 3)
    with pytest.raises(lib.CfdError) as e:
        apply(lib, torch, B, buf, 1, lib.CFD_OP_ALL, lib.CFD_TC_BF16_EXACT)
    assert e.value.status == lib.CFD_ERR_UNSUPPORTED


def test_exact_slices_fp32_uniform_with_iteration(lib, torch):
    """FP32 fields on the uniform decomposition with one hybrid iteration (TMA staging for the
    first halo pass, cp.async with halo columns for the final pass)."""
    NM, N, g = 64, 16, 4
    r = W.rng(909)
    fs = [W.sine_sum(r, 8, 1, 12), W.gaussian(r, 0.1)]
    mesh, dx, exts, buf = uniform(NM, N, g, fs)
    s = lib.cfd_scheme_create(desc("Q13_1_d1"), desc("Q13_1_d2"))
    B = lib.cfd_blocks_bind(s, mesh.n, mesh.dx, mesh.neighbors, g, lib.CFD_F32)
    got = apply(lib, torch, B, buf, 2, lib.CFD_OP_ALL, lib.CFD_TC_BF16_EXACT, 1,
                dtype=np.float32).reshape(mesh.nblocks, 2, 9, N, N, N)
    s1, s2 = oracle_sch("Q13_1_d1"), oracle_sch("Q13_1_d2")
    worst = 0.0
    for q in range(2):
        ref = C.apply_uniform(exts[q].astype(np.float32).astype(np.float64), s1, s2, (dx, dx, dx), N, g, OPS, 1)
        for i, op in enumerate(OPS):
            worst = max(worst, rel_max(got[:, q, i], ref[op].reshape(mesh.nblocks, N, N, N)))
    print("fp32 iterated max rel err", worst)
    assert worst < TOL_EXACT32
