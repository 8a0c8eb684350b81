"""GPU parity of the FP64 banded path (through the C ABI) against the oracle.

Tolerances: FP64 results within 1e-12 relative max error per (field, op);
the ghost exchange is a copy and must be bit-exact; FP32 fields are compared
after rounding the oracle's FP64 result, within one FP32 rounding.
"""
import numpy as np
import pytest

from oracle import cfd as C
from paper_2302_14858_gb300 import workloads as W
from tests.helpers import OPS, desc, oracle_sch, rel_max, wavenumber

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


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


def scheme(lib, kind="Q13_1"):
    return lib.cfd_scheme_create(desc(f"{kind}_d1"), desc(f"{kind}_d2"))


def run_apply(lib, torch, blocks, buf_np, nf, mask, n_iter, prec=0, dtype=np.float64):
    dev = torch.device("cuda", 0)
    fields = torch.from_numpy(np.ascontiguousarray(buf_np.astype(dtype))).to(dev)
    nops = bin(mask).count("1")
    nint = sum(int(n) ** 3 for n in blocks.block_n)
    out = torch.zeros(nint * nf * nops, dtype=fields.dtype, device=dev)
    ws = lib.cfd_apply_workspace(blocks, nf, mask, prec, n_iter)
    work = torch.empty(max(ws, 256), dtype=torch.uint8, device=dev)
    lib.cfd_apply(blocks, fields, nf, mask, prec, n_iter, out, work)
    lib.cfd_sync_status(blocks)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def uniform_case(NM, N, g, fields, seed_shift=0):
    """Global periodic samples -> oracle ext arrays + packed GPU buffer."""
    mesh = W.uniform_mesh(NM, N, g)
    dx = 2 * np.pi / NM
    x = (np.arange(NM) + 0.5) * dx
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    exts = [C.ghost_fill_3d(f(X, Y, Z), N, g) for f in fields]
    nb = mesh.nblocks
    E = N + 2 * g
    buf = np.stack([e.reshape(nb, E, E, E) for e in exts], axis=1).reshape(-1)
    return mesh, dx, exts, buf


def case_fields(seed, n=4):
    r = W.rng(seed)
    out = [W.sine_sum(r, 8, 1, 12), W.gaussian(r, 0.1)]
    while len(out) < n:
        out.append(W.sine_sum(r, 8, 1, 12) if len(out) % 2 == 0 else W.gaussian(r, 0.1))
    return out[:n]


# ------------------------------------------------------------------ ghost exchange


def test_exchange_bit_exact(lib, torch):
    NM, N, g = 32, 8, 4
    mesh = W.uniform_mesh(NM, N, g)
    r = np.random.default_rng(1)
    E = N + 2 * g
    nf = 3
    blocks = r.standard_normal((mesh.nblocks, nf, E, E, E))
    s = scheme(lib)
    B = lib.cfd_blocks_bind(s, mesh.n, mesh.dx, mesh.neighbors, g, lib.CFD_F64)
    t = torch.from_numpy(blocks.reshape(-1).copy()).cuda()
    lib.cfd_exchange_ghosts(B, t, nf)
    torch.cuda.synchronize()
    got = t.cpu().numpy().reshape(mesh.nblocks, nf, E, E, E)
    for q in range(nf):
        want = C.exchange_ghosts([blocks[b, q] for b in range(mesh.nblocks)], mesh.neighbors, N, g)
        for b in range(mesh.nblocks):
            assert np.array_equal(got[b, q], want[b])


def test_exchange_skips_minus_one_and_float32(lib, torch):
    NM, N, g = 32, 16, 4
    mesh = W.uniform_mesh(NM, N, g)
    nbr = mesh.neighbors.copy()
    nbr[0, :5] = -1
    nbr[3, 20:] = -1
    r = np.random.default_rng(2)
    E = N + 2 * g
    blocks = r.standard_normal((mesh.nblocks, 1, E, E, E)).astype(np.float32)
    s = scheme(lib)
    B = lib.cfd_blocks_bind(s, mesh.n, mesh.dx, nbr, g, lib.CFD_F32)
    t = torch.from_numpy(blocks.reshape(-1).copy()).cuda()
    lib.cfd_exchange_ghosts(B, t, 1)
    got = t.cpu().numpy().reshape(mesh.nblocks, E, E, E)
    want = C.exchange_ghosts([blocks[b, 0] for b in range(mesh.nblocks)], nbr, N, g)
    for b in range(mesh.nblocks):
        assert np.array_equal(got[b], want[b])


# ------------------------------------------------------------------ single periodic block (cyclic)


@pytest.mark.parametrize("kind", ["P2", "Q13_1"])
def test_single_block_is_global_scheme(lib, torch, kind):
    """One periodic 32^3 block (its own neighbour): the undecomposed cyclic scheme along every axis."""
    NM = N = 32
    g = 4
    f = W.workload_fields(1)[0]
    mesh, dx, exts, buf = uniform_case(NM, N, g, [f])
    s = scheme(lib, kind)
    B = lib.cfd_blocks_bind(s, mesh.n, mesh.dx, mesh.neighbors, g, lib.CFD_F64)
    mask = lib.CFD_OP_ALL
    got = run_apply(lib, torch, B, buf, 1, mask, 0).reshape(9, N, N, N)
    s1, s2 = oracle_sch(f"{kind}_d1"), oracle_sch(f"{kind}_d2")
    x = (np.arange(NM) + 0.5) * dx
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    fg = f(X, Y, Z)

    def glob(a, sch, arr):
        return np.moveaxis(C.global_periodic(np.moveaxis(arr, a, 0), sch, dx), 0, a)

    want = {"dx": glob(2, s1, fg), "dy": glob(1, s1, fg), "dz": glob(0, s1, fg),
            "dxx": glob(2, s2, fg), "dyy": glob(1, s2, fg), "dzz": glob(0, s2, fg)}
    want["dxy"] = glob(2, s1, glob(1, s1, fg))
    want["dxz"] = glob(2, s1, glob(0, s1, fg))
    want["dyz"] = glob(1, s1, glob(0, s1, fg))
    for i, op in enumerate(OPS):
        assert rel_max(got[i], want[op]) < TOL64, op
    # closed form of the cyclic scheme on the sine sum: each mode scaled by eta~(k_x dx)/dx
    closed = 0.0
    for (kx, ky, kz), A, ph in zip(f.k, f.A, f.phi):
        closed = closed + A * wavenumber(f"{kind}_d1", kx * dx) / dx * np.cos(kx * X + ky * Y + kz * Z + ph)
    assert rel_max(got[0], closed) < 1e-12
    # the continuous derivative differs by the scheme's spectral error at up to ~3 points per wavelength
    assert rel_max(got[0], f.deriv("dx", X, Y, Z)) < 0.05


# ------------------------------------------------------------------ decomposed uniform meshes


@pytest.mark.parametrize("NM,N", [(64, 16), (64, 32), (32, 8)])
@pytest.mark.parametrize("n_iter", [0, 1, 2])
def test_uniform_all_ops_fp64(lib, torch, NM, N, n_iter):
    g = 4
    fields = case_fields(100 + NM + N)
    mesh, dx, exts, buf = uniform_case(NM, N, g, fields)
    s = scheme(lib)
    B = lib.cfd_blocks_bind(s, mesh.n, mesh.dx, mesh.neighbors, g, lib.CFD_F64)
    nf = len(fields)
    got = run_apply(lib, torch, B, buf, nf, lib.CFD_OP_ALL, n_iter).reshape(mesh.nblocks, nf, 9, N, N, N)
    s1, s2 = oracle_sch("Q13_1_d1"), oracle_sch("Q13_1_d2")
    for q in range(nf):
        ref = C.apply_uniform(exts[q], s1, s2, (dx, dx, dx), N, g, OPS, n_iter)
        for i, op in enumerate(OPS):
            want = ref[op].reshape(mesh.nblocks, N, N, N)
            err = rel_max(got[:, q, i], want)
            assert err < TOL64, (q, op, err)


@pytest.mark.parametrize("n_iter", [0, 1])
def test_mixed_one_order_equals_symmetrised(lib, torch, n_iter):
    """cfd_blocks_set_mixed_order(1): d_ij as D_i D_j only matches the oracle's averaged form of
    Sec. "Z4c: system description" to rounding on a uniform decomposition (the block operators of
    different axes commute there); single-axis ops are unchanged bit for bit."""
    NM, N, g = 64, 16, 4
    fields = case_fields(211, 2)
    mesh, dx, exts, buf = uniform_case(NM, N, g, fields)
    s = scheme(lib)
    B = lib.cfd_blocks_bind(s, mesh.n, mesh.dx, mesh.neighbors, g, lib.CFD_F64)
    both = run_apply(lib, torch, B, buf, 2, lib.CFD_OP_ALL, n_iter).reshape(mesh.nblocks, 2, 9, N, N, N)
    lib.cfd_blocks_set_mixed_order(B, True)
    one = run_apply(lib, torch, B, buf, 2, lib.CFD_OP_ALL, n_iter).reshape(mesh.nblocks, 2, 9, N, N, N)
    assert np.array_equal(one[:, :, :6], both[:, :, :6])
    s1, s2 = oracle_sch("Q13_1_d1"), oracle_sch("Q13_1_d2")
    for q in range(2):
        ref = C.apply_uniform(exts[q], s1, s2, (dx, dx, dx), N, g, OPS, n_iter)
        for i, op in enumerate(OPS):
            assert rel_max(one[:, q, i], ref[op].reshape(mesh.nblocks, N, N, N)) < TOL64, op
    lib.cfd_blocks_set_mixed_order(B, False)
    again = run_apply(lib, torch, B, buf, 2, lib.CFD_OP_ALL, n_iter).reshape(mesh.nblocks, 2, 9, N, N, N)
    assert np.array_equal(again, both)


def test_mixed_one_order_refused_without_face_neighbours(lib):
    mesh = mini_box_in_box()
    s = scheme(lib)
    B = lib.cfd_blocks_bind(s, mesh.n, mesh.dx, mesh.neighbors, mesh.g, lib.CFD_F64)
    with pytest.raises(lib.CfdError) as e:
        lib.cfd_blocks_set_mixed_order(B, True)
    assert e.value.status == lib.CFD_ERR_UNSUPPORTED


def test_op_subset_order_and_padé(lib, torch):
    """A subset mask writes only those ops, in bit order; Padé P^1_2 with its closure."""
    NM, N, g = 32, 16, 4
    fields = case_fields(7, 2)
    mesh, dx, exts, buf = uniform_case(NM, N, g, fields)
    s = scheme(lib, "P2")
    B = lib.cfd_blocks_bind(s, mesh.n, mesh.dx, mesh.neighbors, g, lib.CFD_F64)
    ops = ["dy", "dzz", "dxz"]
    mask = lib.op_mask(ops)
    got = run_apply(lib, torch, B, buf, 2, mask, 1).reshape(mesh.nblocks, 2, 3, N, N, N)
    s1, s2 = oracle_sch("P2_d1"), oracle_sch("P2_d2")
    for q in range(2):
        ref = C.apply_uniform(exts[q], s1, s2, (dx, dx, dx), N, g, ops, 1)
        for i, op in enumerate(ops):
            assert rel_max(got[:, q, i], ref[op].reshape(mesh.nblocks, N, N, N)) < TOL64


# ------------------------------------------------------------------ uneven sizes, FP32, analytic ghosts


def mini_box_in_box(g=4):
    """4^3 coarse blocks of 8^3 (minus the refined octant) + 2^3 fine blocks of 16^3 on [0, 2pi)^3."""
    nc = 4
    ns, origins, ds = [], [], []
    ci, fi = {}, {}
    for bz in range(nc):
        for by in range(nc):
            for bx in range(nc):
                if bx < 2 and by < 2 and bz < 2:
                    continue
                ci[(bz, by, bx)] = len(ns)
                ns.append(8)
                origins.append((bx * 8, by * 8, bz * 8))
                ds.append(2 * np.pi / 32)
    for bz in range(2):
        for by in range(2):
            for bx in range(2):
                fi[(bz, by, bx)] = len(ns)
                ns.append(16)
                origins.append((bx * 16, by * 16, bz * 16))
                ds.append(np.pi / 32)
    nbr = np.full((len(ns), 26), -1, np.int32)
    for (bz, by, bx), b in ci.items():
        for r, (dz, dy, dxx) in enumerate(W.DIRS):
            nbr[b, r] = ci.get(((bz + dz) % nc, (by + dy) % nc, (bx + dxx) % nc), -1)
    for (bz, by, bx), b in fi.items():
        for r, (dz, dy, dxx) in enumerate(W.DIRS):
            nbr[b, r] = fi.get((bz + dz, by + dy, bx + dxx), -1)
    dx = np.repeat(np.asarray(ds)[:, None], 3, 1)
    return W.Mesh(np.asarray(ns), np.asarray(origins), dx, nbr, g)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_uneven_blocks_analytic_ghosts(lib, torch, dtype):
    mesh = mini_box_in_box()
    g = mesh.g
    fields = W.workload_fields(4)[:3]
    per_block = W.sample(mesh, fields, dtype=dtype)
    buf = W.pack(per_block)
    s = scheme(lib)
    B = lib.cfd_blocks_bind(s, mesh.n, mesh.dx, mesh.neighbors, g,
                            lib.CFD_F64 if dtype == np.float64 else lib.CFD_F32)
    nf = len(fields)
    out = run_apply(lib, torch, B, buf, nf, lib.CFD_OP_ALL, 0, dtype=dtype)
    got = W.unpack(out, mesh, nf, interior=True, nops=9)
    s1, s2 = oracle_sch("Q13_1_d1"), oracle_sch("Q13_1_d2")
    worst = 0.0
    for q in range(nf):
        for i, op in enumerate(OPS):
            want = [C.apply_block(per_block[b][q].astype(np.float64), s1, s2, mesh.dx[b], int(mesh.n[b]), g, (op,))[op]
                    for b in range(mesh.nblocks)]
            wmax = max(np.abs(w).max() for w in want)
            err = max(np.abs(got[b][q, i].astype(np.float64) - want[b]).max() for b in range(mesh.nblocks)) / wmax
            worst = max(worst, err)
    tol = TOL64 if dtype == np.float64 else 6e-8
    assert worst < tol


def test_iteration_rejected_with_open_faces(lib, torch):
    mesh = mini_box_in_box()
    s = scheme(lib)
    B = lib.cfd_blocks_bind(s, mesh.n, mesh.dx, mesh.neighbors, mesh.g, lib.CFD_F64)
    buf = np.zeros(sum((int(n) + 8) ** 3 for n in mesh.n))
    with pytest.raises(lib.CfdError) as e:
        run_apply(lib, torch, B, buf, 1, lib.CFD_OP_DX, 1)
    assert e.value.status == lib.CFD_ERR_UNSUPPORTED


# ------------------------------------------------------------------ RK4 wave driver


@pytest.mark.parametrize("n_iter", [0, 1])
def test_wave_rk4_steps(lib, torch, n_iter):
    NM, N, g = 32, 8, 4
    pw = W.plane_waves(11, 4, 6.0)
    dx = 2 * np.pi / NM
    x = (np.arange(NM) + 0.5) * dx
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    phi0, K0 = pw.phi_at(0.0, X, Y, Z), pw.K_at(0.0, X, Y, Z)
    mesh = W.uniform_mesh(NM, N, g)
    s = scheme(lib)
    B = lib.cfd_blocks_bind(s, mesh.n, mesh.dx, mesh.neighbors, g, lib.CFD_F64)
    E = N + 2 * g
    pe = C.ghost_fill_3d(phi0, N, g).reshape(mesh.nblocks, E, E, E)
    ke = C.ghost_fill_3d(K0, N, g).reshape(mesh.nblocks, E, E, E)
    tp = torch.from_numpy(pe.reshape(-1).copy()).cuda()
    tk = torch.from_numpy(ke.reshape(-1).copy()).cuda()
    ws = lib.cfd_wave_workspace(B, 0, n_iter)
    work = torch.empty(ws, dtype=torch.uint8, device="cuda")
    dt = 0.25 * dx
    s2 = oracle_sch("Q13_1_d2")
    p, k = phi0, K0
    for _ in range(3):
        lib.cfd_wave_rk_step(B, tp, tk, dt, 0, n_iter, work)
        p, k = C.wave_rk4_step(p, k, dt, s2, (dx, dx, dx), N, g, n_iter)
    lib.cfd_sync_status(B)
    gp = tp.cpu().numpy().reshape(mesh.nblocks, E, E, E)[:, g:g + N, g:g + N, g:g + N]
    gk = tk.cpu().numpy().reshape(mesh.nblocks, E, E, E)[:, g:g + N, g:g + N, g:g + N]
    nb = NM // N
    gp = C.blocks_to_global(gp.reshape(nb, nb, nb, N, N, N))
    gk = C.blocks_to_global(gk.reshape(nb, nb, nb, N, N, N))
    assert rel_max(gp, p) < TOL64
    assert rel_max(gk, k) < TOL64
