"""GPU parity of the biased (upwind) FP64 path through the C ABI against oracle/biased.py.

Biased derivatives (Eq. closure_left_X and its mirror, Eq. iter_left_X), the
single-block cyclic case, FP32 fields and the upwinded shift-advection term
(Eq. biasderapproxadv).  Tolerances: FP64 within 1e-12 relative max error per
(field, axis); FP32 fields within 2e-6 of the oracle's FP64 result on the same
(rounded) input.
"""
import numpy as np
import pytest

from oracle import biased as B
from oracle import cfd as C
from tests.helpers import SCHEMES, desc, rel_max
from tests.test_gpu_banded import case_fields, uniform_case

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
AXES = ("x", "y", "z")


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


def biased_of(name):
    e = SCHEMES[name]
    return B.Biased(e["a"], e["lo"], tuple(e["rhs"]), e["c_sup"], e["c_lo"], tuple(e["closure"]), e["kc"])


def bind(lib, name, mesh, g, dtype):
    s = lib.cfd_scheme_create(desc("Q13_1_d1"), None)
    lib.cfd_scheme_set_biased(s, SCHEMES[name])
    return lib.cfd_blocks_bind(s, mesh.n, mesh.dx, mesh.neighbors, g, dtype)


TOL_TC = 1e-7       # exact digit slices on the tensor cores (the centred path's contract)


def run_biased(lib, torch, blocks, buf, nf, mask, side, n_iter, dtype=np.float64, prec=0):
    dev = torch.device("cuda", 0)
    fields = torch.from_numpy(np.ascontiguousarray(buf.astype(dtype))).to(dev)
    nops = bin(mask).count("1")
    nint = sum(int(n) ** 3 for n in blocks.block_n)
    out = torch.zeros(nint * nf * nops, dtype=fields.dtype, device=dev)
    ws = lib.cfd_biased_workspace(blocks, nf, prec, n_iter)
    work = torch.empty(max(ws, 256), dtype=torch.uint8, device=dev)
    lib.cfd_apply_biased(blocks, fields, nf, mask, side, prec, n_iter, out, work)
    lib.cfd_sync_status(blocks)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def check_biased(lib, torch, name, NM, N, g, side, n_iter, nf=2, seed=11, prec=0):
    fields = case_fields(seed, nf)
    mesh, dx, exts, buf = uniform_case(NM, N, g, fields)
    blocks = bind(lib, name, mesh, g, lib.CFD_F64)
    got = run_biased(lib, torch, blocks, buf, nf, lib.CFD_OP_DX | lib.CFD_OP_DY | lib.CFD_OP_DZ, side, n_iter,
                     prec=prec)
    got = got.reshape(mesh.nblocks, nf, 3, N, N, N)
    b = biased_of(name)
    tol = TOL64 if prec == 0 else TOL_TC
    for q in range(nf):
        want = B.biased_uniform(exts[q], b, side, (dx, dx, dx), N, g, AXES, n_iter)
        for i, c in enumerate(AXES):
            w = want[c].reshape(mesh.nblocks, N, N, N)
            assert rel_max(got[:, q, i], w) < tol, (name, side, n_iter, q, c, rel_max(got[:, q, i], w))


@pytest.mark.parametrize("name", ["X2_d1", "Q1034_1_d1"])
@pytest.mark.parametrize("side", [1, -1])
@pytest.mark.parametrize("NM,N,n_iter", [(64, 16, 0), (64, 16, 1), (64, 32, 1), (64, 16, 2)])
def test_biased_parity_tensor_cores(lib, torch, name, side, NM, N, n_iter):
    """The dense biased operators (closed, iterated with one-sided halo columns) on the tensor
    cores, exact digit slices."""
    check_biased(lib, torch, name, NM, N, 4, side, n_iter, prec=2)


@pytest.mark.parametrize("side", [1, -1])
def test_biased_tensor_cores_bf16x3(lib, torch, side):
    """BF16 hi/lo (3 products) on the same operators: the lower-precision measured mode
    (5e-4 measured here; bound 5e-3, as the centred path keeps this mode's bound separate from
    the FP64-grade contract)."""
    NM, N, g = 64, 16, 4
    fields = case_fields(11, 1)
    mesh, dx, exts, buf = uniform_case(NM, N, g, fields)
    blocks = bind(lib, "X2_d1", mesh, g, lib.CFD_F64)
    got = run_biased(lib, torch, blocks, buf, 1, lib.CFD_OP_DX, side, 1, prec=1).reshape(mesh.nblocks, N, N, N)
    want = B.biased_uniform(exts[0], biased_of("X2_d1"), side, (dx, dx, dx), N, g, ("x",), 1)["x"]
    assert rel_max(got, want.reshape(mesh.nblocks, N, N, N)) < 5e-3


@pytest.mark.parametrize("name", ["X1_d1", "X2_d1", "Q1034_1_d1"])
@pytest.mark.parametrize("side", [1, -1])
@pytest.mark.parametrize("n_iter", [0, 1, 2])
def test_biased_parity_16(lib, torch, name, side, n_iter):
    """64^3 as 4^3 blocks of 16^3, ng = 4: closed block systems and their iteration."""
    check_biased(lib, torch, name, 64, 16, 4, side, n_iter)


@pytest.mark.parametrize("NM,N", [(64, 32), (32, 8)])
@pytest.mark.parametrize("side", [1, -1])
def test_biased_parity_other_sizes(lib, torch, NM, N, side):
    """Block sizes 32 and 8 (several tiles of pencils; 8 leaves half a thread block idle)."""
    check_biased(lib, torch, "X2_d1", NM, N, 4, side, 1)


@pytest.mark.parametrize("side", [1, -1])
def test_biased_parity_wide_stencil(lib, torch, side):
    """X_3 (interior offsets -5..5, closure to 6) with ng = 6."""
    check_biased(lib, torch, "X3_d1", 64, 16, 6, side, 1)


@pytest.mark.parametrize("side", [1, -1])
def test_single_block_is_the_cyclic_scheme(lib, torch, side):
    """A 32^3 block that is its own neighbour: the undecomposed periodic biased scheme."""
    NM = N = 32
    g = 4
    fields = case_fields(5, 1)
    mesh, dx, exts, buf = uniform_case(NM, N, g, fields)
    blocks = bind(lib, "Q1034_1_d1", mesh, g, lib.CFD_F64)
    b = biased_of("Q1034_1_d1")
    fg = exts[0][0, 0, 0][g:g + N, g:g + N, g:g + N]
    for prec, tol in ((0, TOL64), (2, TOL_TC)):
        got = run_biased(lib, torch, blocks, buf, 1, lib.CFD_OP_DX | lib.CFD_OP_DY | lib.CFD_OP_DZ, side, 2,
                         prec=prec)
        got = got.reshape(3, N, N, N)
        for i, ax in enumerate((2, 1, 0)):
            want = np.moveaxis(B.global_periodic(np.moveaxis(fg, ax, 0), b, side, dx), 0, ax)
            assert rel_max(got[i], want) < tol, (prec, i)


def test_iteration_reaches_the_global_scheme(lib, torch):
    """Five iterations of Eq. iter_left_X on 16^3 blocks (each one damps the closure error by
    about |a|^(N+kc) = 1.4e-3): the global periodic result."""
    NM, N, g = 64, 16, 4
    fields = case_fields(3, 1)
    mesh, dx, exts, buf = uniform_case(NM, N, g, fields)
    blocks = bind(lib, "X2_d1", mesh, g, lib.CFD_F64)
    b = biased_of("X2_d1")
    x = (np.arange(NM) + 0.5) * dx
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    fg = fields[0](X, Y, Z)
    for side in (1, -1):
        got = run_biased(lib, torch, blocks, buf, 1, lib.CFD_OP_DX, side, 5).reshape(mesh.nblocks, N, N, N)
        want = np.moveaxis(B.global_periodic(np.moveaxis(fg, 2, 0), b, side, dx), 0, 2)
        assert rel_max(C.blocks_to_global(got.reshape(4, 4, 4, N, N, N)), want) < 1e-13
        got0 = run_biased(lib, torch, blocks, buf, 1, lib.CFD_OP_DX, side, 0).reshape(mesh.nblocks, N, N, N)
        assert rel_max(C.blocks_to_global(got0.reshape(4, 4, 4, N, N, N)), want) > 1e-9


def test_float32_fields(lib, torch):
    NM, N, g = 64, 16, 4
    fields = case_fields(9, 2)
    mesh, dx, exts, buf = uniform_case(NM, N, g, fields)
    buf32 = buf.astype(np.float32)
    blocks = bind(lib, "X2_d1", mesh, g, lib.CFD_F32)
    got = run_biased(lib, torch, blocks, buf32, 2, lib.CFD_OP_DX | lib.CFD_OP_DZ, -1, 1, np.float32)
    got = got.reshape(mesh.nblocks, 2, 2, N, N, N).astype(np.float64)
    b = biased_of("X2_d1")
    E = N + 2 * g
    for q in range(2):
        ext = buf32.reshape(mesh.nblocks, 2, E, E, E)[:, q].astype(np.float64).reshape(exts[q].shape)
        want = B.biased_uniform(ext, b, -1, (dx, dx, dx), N, g, ("x", "z"), 1)
        for i, c in enumerate(("x", "z")):
            assert rel_max(got[:, q, i], want[c].reshape(mesh.nblocks, N, N, N)) < 2e-6


def shift_fields():
    """Shift components with both signs inside every block."""
    return [lambda X, Y, Z: np.cos(X + 2 * Z) + 0.1,
            lambda X, Y, Z: np.sin(Y - X),
            lambda X, Y, Z: 0.5 * np.cos(3 * Y) * np.sin(Z)]


@pytest.mark.parametrize("name,g", [("X2_d1", 4), ("Q1034_1_d1", 4)])
@pytest.mark.parametrize("n_iter", [0, 1, 2])
@pytest.mark.parametrize("shift", ["mixed", "one_sign"])
@pytest.mark.parametrize("prec", [0, 2])
def test_advect_parity(lib, torch, name, g, n_iter, shift, prec):
    """out = sum_i beta^i_+ D_i[S+] f + beta^i_- D_i[S-] f on 4^3 blocks of 16^3, 3 fields.
    "one_sign": beta^x > 0, beta^y = 0, beta^z < 0 everywhere (pencils that need one side, or none)."""
    NM, N, nf = 64, 16, 3
    fields = case_fields(21, nf)
    mesh, dx, exts, buf = uniform_case(NM, N, g, fields)
    sf = shift_fields() if shift == "mixed" else [lambda X, Y, Z: 0.3 + 0.1 * np.sin(Y),
                                                  lambda X, Y, Z: 0.0 * X,
                                                  lambda X, Y, Z: -0.7 + 0.2 * np.cos(X)]
    _, _, bexts, bbuf = uniform_case(NM, N, g, sf)
    blocks = bind(lib, name, mesh, g, lib.CFD_F64)
    dev = torch.device("cuda", 0)
    f_t = torch.from_numpy(buf).to(dev)
    b_t = torch.from_numpy(bbuf).to(dev)
    out = torch.zeros(mesh.nblocks * nf * N ** 3, dtype=torch.float64, device=dev)
    ws = lib.cfd_biased_workspace(blocks, nf, prec, n_iter)
    work = torch.empty(max(ws, 256), dtype=torch.uint8, device=dev)
    lib.cfd_advect(blocks, f_t, nf, b_t, prec, n_iter, out, work)
    lib.cfd_sync_status(blocks)
    got = out.cpu().numpy().reshape(mesh.nblocks, nf, N, N, N)
    I = slice(g, g + N)
    beta = [e[:, :, :, I, I, I] for e in bexts]
    b = biased_of(name)
    for q in range(nf):
        want = B.advect_uniform(exts[q], beta, b, (dx, dx, dx), N, g, n_iter).reshape(mesh.nblocks, N, N, N)
        assert rel_max(got[:, q], want) < (TOL64 if prec == 0 else TOL_TC)


def test_advect_many_fields_tc(lib, torch):
    """Six fields on the tensor cores (the blend handles fields in groups of four, the second
    group partial): every field against the FP64 banded path, the first and last against the oracle."""
    NM, N, g, nf, name = 64, 16, 4, 6, "X2_d1"
    fields = case_fields(23, nf)
    mesh, dx, exts, buf = uniform_case(NM, N, g, fields)
    _, _, bexts, bbuf = uniform_case(NM, N, g, shift_fields())
    blocks = bind(lib, name, mesh, g, lib.CFD_F64)
    dev = torch.device("cuda", 0)
    f_t = torch.from_numpy(buf).to(dev)
    b_t = torch.from_numpy(bbuf).to(dev)
    outs = []
    for prec in (0, 2):
        out = torch.zeros(mesh.nblocks * nf * N ** 3, dtype=torch.float64, device=dev)
        ws = lib.cfd_biased_workspace(blocks, nf, prec, 1)
        work = torch.empty(max(ws, 256), dtype=torch.uint8, device=dev)
        lib.cfd_advect(blocks, f_t, nf, b_t, prec, 1, out, work)
        lib.cfd_sync_status(blocks)
        outs.append(out.cpu().numpy().reshape(mesh.nblocks, nf, N, N, N))
    assert rel_max(outs[1], outs[0]) < TOL_TC
    I = slice(g, g + N)
    beta = [e[:, :, :, I, I, I] for e in bexts]
    b = biased_of(name)
    for q in (0, nf - 1):
        want = B.advect_uniform(exts[q], beta, b, (dx, dx, dx), N, g, 1).reshape(mesh.nblocks, N, N, N)
        assert rel_max(outs[0][:, q], want) < TOL64
        assert rel_max(outs[1][:, q], want) < TOL_TC


@pytest.mark.parametrize("prec", [0, 2])
def test_advect_float32_fields(lib, torch, prec):
    """FP32 fields and shift (5 fields: the tensor-core blend's second group of four is partial),
    within 2e-6 of the oracle's FP64 result on the same rounded inputs."""
    NM, N, g, nf, name = 64, 16, 4, 5, "X2_d1"
    fields = case_fields(27, nf)
    mesh, dx, exts, buf = uniform_case(NM, N, g, fields)
    _, _, bexts, bbuf = uniform_case(NM, N, g, shift_fields())
    buf32, bbuf32 = buf.astype(np.float32), bbuf.astype(np.float32)
    blocks = bind(lib, name, mesh, g, lib.CFD_F32)
    dev = torch.device("cuda", 0)
    f_t = torch.from_numpy(buf32).to(dev)
    b_t = torch.from_numpy(bbuf32).to(dev)
    out = torch.zeros(mesh.nblocks * nf * N ** 3, dtype=torch.float32, device=dev)
    ws = lib.cfd_biased_workspace(blocks, nf, prec, 1)
    work = torch.empty(max(ws, 256), dtype=torch.uint8, device=dev)
    lib.cfd_advect(blocks, f_t, nf, b_t, prec, 1, out, work)
    lib.cfd_sync_status(blocks)
    got = out.cpu().numpy().astype(np.float64).reshape(mesh.nblocks, nf, N, N, N)
    E = N + 2 * g
    I = slice(g, g + N)
    b32 = bbuf32.reshape(mesh.nblocks, 3, E, E, E).astype(np.float64)
    beta = [b32[:, i].reshape(bexts[i].shape)[:, :, :, I, I, I] for i in range(3)]
    b = biased_of(name)
    for q in range(nf):
        ext = buf32.reshape(mesh.nblocks, nf, E, E, E)[:, q].astype(np.float64).reshape(exts[q].shape)
        want = B.advect_uniform(ext, beta, b, (dx, dx, dx), N, g, 1).reshape(mesh.nblocks, N, N, N)
        assert rel_max(got[:, q], want) < 2e-6


def test_rejections(lib, torch):
    NM, N, g = 32, 16, 4
    fields = case_fields(1, 1)
    mesh, dx, exts, buf = uniform_case(NM, N, g, fields)
    dev = torch.device("cuda", 0)
    f_t = torch.from_numpy(buf).to(dev)
    out = torch.zeros(mesh.nblocks * N ** 3 * 3, dtype=torch.float64, device=dev)
    # no biased scheme bound
    s = lib.cfd_scheme_create(desc("Q13_1_d1"), None)
    B0 = lib.cfd_blocks_bind(s, mesh.n, mesh.dx, mesh.neighbors, g, lib.CFD_F64)
    with pytest.raises(lib.CfdError) as e:
        lib.cfd_apply_biased(B0, f_t, 1, lib.CFD_OP_DX, 1, 0, 0, out)
    assert e.value.status == lib.CFD_ERR_ARG
    blocks = bind(lib, "X2_d1", mesh, g, lib.CFD_F64)
    with pytest.raises(lib.CfdError) as e:                       # TF32 is not built
        lib.cfd_apply_biased(blocks, f_t, 1, lib.CFD_OP_DX, 1, lib.CFD_TC_TF32, 0, out)
    assert e.value.status == lib.CFD_ERR_UNSUPPORTED
    with pytest.raises(lib.CfdError) as e:                       # tensor cores need their workspace
        lib.cfd_apply_biased(blocks, f_t, 1, lib.CFD_OP_DX, 1, lib.CFD_TC_BF16_EXACT, 0, out, None)
    assert e.value.status == lib.CFD_ERR_ARG
    with pytest.raises(lib.CfdError) as e:                       # side must be +-1
        lib.cfd_apply_biased(blocks, f_t, 1, lib.CFD_OP_DX, 0, 0, 0, out)
    assert e.value.status == lib.CFD_ERR_ARG
    with pytest.raises(lib.CfdError) as e:                       # second-degree ops are not biased
        lib.cfd_apply_biased(blocks, f_t, 1, lib.CFD_OP_DXX, 1, 0, 0, out)
    assert e.value.status == lib.CFD_ERR_ARG
    with pytest.raises(lib.CfdError) as e:                       # iteration needs the halo workspace
        lib.cfd_apply_biased(blocks, f_t, 1, lib.CFD_OP_DX, 1, 0, 1, out, None)
    assert e.value.status == lib.CFD_ERR_ARG
    # ghost width outside the compiled windows
    mesh5 = uniform_case(NM, N, 5, fields)[0]
    s5 = lib.cfd_scheme_create(desc("Q13_1_d1"), None)
    lib.cfd_scheme_set_biased(s5, SCHEMES["X2_d1"])
    B5 = lib.cfd_blocks_bind(s5, mesh5.n, mesh5.dx, mesh5.neighbors, 5, lib.CFD_F64)
    with pytest.raises(lib.CfdError) as e:
        lib.cfd_apply_biased(B5, f_t, 1, lib.CFD_OP_DX, 1, 0, 0, out)
    assert e.value.status == lib.CFD_ERR_UNSUPPORTED
    # bad descriptors are refused on the host
    bad = dict(SCHEMES["X2_d1"], a=1.2)
    with pytest.raises(lib.CfdError):
        lib.cfd_scheme_set_biased(s5, bad)
    bad = dict(SCHEMES["X2_d1"], kc=0)
    with pytest.raises(lib.CfdError):
        lib.cfd_scheme_set_biased(s5, bad)
    torch.cuda.synchronize()


@pytest.mark.parametrize("prec,n_iter", [(0, 0), (0, 1), (2, 1)])
def test_shifted_wave_lsrk_parity(lib, torch, prec, n_iter):
    """Two 2S steps of the shifted wave system (Eq. toyShiftWaveEqnSys, flat background) with a
    mixed-sign shift field and Kreiss-Oliger dissipation vs the oracle."""
    from oracle import timestep as T
    from paper_2302_14858_gb300 import workloads as W
    from tests.helpers import oracle_sch
    NM, N, g, sigma, r = 64, 16, 4, 0.04, 4
    pw = W.plane_waves(19, 4, 10.0)
    dx = 2 * np.pi / NM
    x = (np.arange(NM) + 0.5) * dx
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    phi0 = pw.phi_at(0.0, X, Y, Z) + 0.05 * np.cos(11 * X - 9 * Y + 7 * Z)
    K0 = pw.K_at(0.0, X, Y, Z)
    beta_g = [f(X, Y, Z) for f in shift_fields()]
    mesh, _, _, bbuf = uniform_case(NM, N, g, shift_fields())
    s = lib.cfd_scheme_create(desc("Q13_1_d1"), desc("Q13_1_d2"))
    lib.cfd_scheme_set_biased(s, SCHEMES["X2_d1"])
    Bk = lib.cfd_blocks_bind(s, mesh.n, mesh.dx, mesh.neighbors, g, lib.CFD_F64)
    E = N + 2 * g
    tp = torch.from_numpy(C.ghost_fill_3d(phi0, N, g).reshape(-1).copy()).cuda()
    tk = torch.from_numpy(C.ghost_fill_3d(K0, N, g).reshape(-1).copy()).cuda()
    tb = torch.from_numpy(bbuf).cuda()
    work = torch.empty(lib.cfd_shifted_wave_workspace(Bk, prec, n_iter), dtype=torch.uint8, device="cuda")
    coef = T.lsrk2s_rk4_float()
    dt = 0.25 * dx
    s2 = oracle_sch("Q13_1_d2")
    b = biased_of("X2_d1")
    p, k = phi0, K0
    for _ in range(2):
        lib.cfd_shifted_wave_lsrk_step(Bk, tp, tk, tb, dt, coef, sigma, r, prec, n_iter, work)
        p, k = T.shifted_wave_lsrk_step(p, k, beta_g, dt, coef, s2, b, (dx, dx, dx), N, g, n_iter, sigma, r)
    lib.cfd_sync_status(Bk)
    nb = NM // N
    I = slice(g, g + N)
    gp = C.blocks_to_global(tp.cpu().numpy().reshape(mesh.nblocks, E, E, E)[:, I, I, I].reshape(nb, nb, nb, N, N, N))
    gk = C.blocks_to_global(tk.cpu().numpy().reshape(mesh.nblocks, E, E, E)[:, I, I, I].reshape(nb, nb, nb, N, N, N))
    tol = 1e-12 if prec == 0 else 1e-7
    assert rel_max(gp, p) < tol, rel_max(gp, p)
    assert rel_max(gk, k) < tol, rel_max(gk, k)
    # the shift terms are visible: the unshifted step differs well beyond the tolerance
    p0, _ = T.wave_lsrk_step(phi0, K0, dt, coef, s2, (dx, dx, dx), N, g, n_iter, sigma, r)
    p1, _ = T.shifted_wave_lsrk_step(phi0, K0, beta_g, dt, coef, s2, b, (dx, dx, dx), N, g, n_iter, sigma, r)
    assert rel_max(p0, p1) > 1e-3


def test_shifted_wave_rejections(lib, torch):
    from oracle import timestep as T
    NM, N, g = 32, 16, 4
    mesh, _, _, bbuf = uniform_case(NM, N, g, shift_fields())
    s = lib.cfd_scheme_create(desc("Q13_1_d1"), desc("Q13_1_d2"))        # no biased scheme
    Bk = lib.cfd_blocks_bind(s, mesh.n, mesh.dx, mesh.neighbors, g, lib.CFD_F64)
    E = N + 2 * g
    t = torch.zeros(mesh.nblocks * E ** 3, dtype=torch.float64, device="cuda")
    tb = torch.from_numpy(bbuf).cuda()
    work = torch.empty(lib.cfd_shifted_wave_workspace(Bk, 0, 0), dtype=torch.uint8, device="cuda")
    with pytest.raises(lib.CfdError) as e:
        lib.cfd_shifted_wave_lsrk_step(Bk, t, t.clone(), tb, 0.01, T.lsrk2s_rk4_float(), 0.0, 4, 0, 0, work)
    assert e.value.status == lib.CFD_ERR_ARG
    torch.cuda.synchronize()


@pytest.mark.parametrize("prec,n_iter", [(0, 0), (0, 1), (2, 1)])
def test_advect_lsrk_parity(lib, torch, prec, n_iter):
    """Two 2S steps of u_t = beta . grad u + KO for two fields with a mixed-sign shift vs the oracle."""
    from oracle import timestep as T
    NM, N, g, sigma, r, nf = 64, 16, 4, 0.04, 4, 2
    fields = case_fields(31, nf)
    mesh, dx, exts, buf = uniform_case(NM, N, g, fields)
    x = (np.arange(NM) + 0.5) * dx
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    beta_g = [f(X, Y, Z) for f in shift_fields()]
    _, _, _, bbuf = uniform_case(NM, N, g, shift_fields())
    Bk = bind(lib, "X2_d1", mesh, g, lib.CFD_F64)
    tu = torch.from_numpy(buf.copy()).cuda()
    tb = torch.from_numpy(bbuf).cuda()
    work = torch.empty(lib.cfd_advect_lsrk_workspace(Bk, nf, prec, n_iter), dtype=torch.uint8, device="cuda")
    coef = T.lsrk2s_rk4_float()
    dt = 0.3 * dx
    b = biased_of("X2_d1")
    us = [f(X, Y, Z) for f in fields]
    for _ in range(2):
        lib.cfd_advect_lsrk_step(Bk, tu, nf, tb, dt, coef, sigma, r, prec, n_iter, work)
        us = [T.advect_lsrk_step(u, beta_g, dt, coef, b, (dx, dx, dx), N, g, n_iter, sigma, r) for u in us]
    lib.cfd_sync_status(Bk)
    E = N + 2 * g
    nb = NM // N
    I = slice(g, g + N)
    got = tu.cpu().numpy().reshape(mesh.nblocks, nf, E, E, E)[:, :, I, I, I]
    tol = 1e-12 if prec == 0 else 1e-7
    for q in range(nf):
        gq = C.blocks_to_global(got[:, q].reshape(nb, nb, nb, N, N, N))
        assert rel_max(gq, us[q]) < tol, (q, rel_max(gq, us[q]))



@pytest.mark.parametrize("side", [1, -1])
def test_biased_uneven_blocks_analytic_ghosts(lib, torch, side):
    """Blocks of 8^3 and 16^3 whose ghosts at the size interface are sampled from the analytic
    field (neighbour -1): closed biased systems per block; the tensor cores refuse the 8^3 group."""
    from paper_2302_14858_gb300 import workloads as W
    from tests.test_gpu_banded import mini_box_in_box
    mesh = mini_box_in_box()
    g = mesh.g
    fields = W.workload_fields(4)[:2]
    per_block = W.sample(mesh, fields)
    buf = W.pack(per_block)
    Bk = bind(lib, "X2_d1", mesh, g, lib.CFD_F64)
    mask = lib.CFD_OP_DX | lib.CFD_OP_DY | lib.CFD_OP_DZ
    out = run_biased(lib, torch, Bk, buf, 2, mask, side, 0)
    got = W.unpack(out, mesh, 2, interior=True, nops=3)
    b_ = biased_of("X2_d1")
    worst = 0.0
    for q in range(2):
        for i, c in enumerate(AXES):
            want = [B.biased_uniform(per_block[b][q][None, None, None], b_, side, mesh.dx[b], int(mesh.n[b]), g,
                                     (c,), 0)[c][0, 0, 0] for b in range(mesh.nblocks)]
            wmax = max(np.abs(w).max() for w in want)
            worst = max(worst, max(np.abs(got[b][q, i] - want[b]).max() for b in range(mesh.nblocks)) / wmax)
    assert worst < TOL64
    with pytest.raises(lib.CfdError) as e:
        run_biased(lib, torch, Bk, buf, 2, mask, side, 0, prec=2)
    assert e.value.status == lib.CFD_ERR_UNSUPPORTED


def test_biased_float32_tensor_cores(lib, torch):
    """FP32 fields through the dense biased operators (exact slices, FP32 outputs)."""
    NM, N, g = 64, 16, 4
    fields = case_fields(13, 1)
    mesh, dx, exts, buf = uniform_case(NM, N, g, fields)
    buf32 = buf.astype(np.float32)
    blocks = bind(lib, "Q1034_1_d1", mesh, g, lib.CFD_F32)
    got = run_biased(lib, torch, blocks, buf32, 1, lib.CFD_OP_DY, 1, 1, np.float32, prec=2)
    got = got.reshape(mesh.nblocks, N, N, N).astype(np.float64)
    E = N + 2 * g
    ext = buf32.reshape(mesh.nblocks, E, E, E).astype(np.float64).reshape(exts[0].shape)
    want = B.biased_uniform(ext, biased_of("Q1034_1_d1"), 1, (dx, dx, dx), N, g, ("y",), 1)["y"]
    assert rel_max(got, want.reshape(mesh.nblocks, N, N, N)) < 2e-6


@pytest.mark.parametrize("name,g", [("X1_d1", 4), ("X3_d1", 6)])
@pytest.mark.parametrize("side", [1, -1])
def test_biased_tensor_cores_other_widths(lib, torch, name, g, side):
    """X_1 (interior -3..3) and X_3 (-5..5, closure to 6, ng = 6: K = N + 2g + 4 = 48 for 32^3)
    through the dense biased operators with one iteration."""
    check_biased(lib, torch, name, 64, 32 if name == "X3_d1" else 16, g, side, 1, nf=1, prec=2)


def mini_two_sizes(g=4):
    """4^3 coarse blocks of 16^3 on [0, 2pi)^3 minus the octant [0, pi)^3, which holds 2^3 fine
    blocks of 32^3 at half the spacing; ghosts facing the other size are the caller's (-1)."""
    from paper_2302_14858_gb300 import workloads as W
    nc = 4
    ns, origins, ds = [], [], []
    ci, fi = {}, {}
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
    dx = np.repeat(np.asarray(ds)[:, None], 3, 1)
    return W.Mesh(np.asarray(ns), np.asarray(origins), dx, nbr, g)


@pytest.mark.parametrize("prec", [0, 2])
def test_advect_two_block_sizes_analytic_ghosts(lib, torch, prec):
    """Upwinded advection on blocks of 16^3 and 32^3 (analytic ghosts at the size interface,
    closures only) on both arithmetics, against the oracle block by block."""
    from paper_2302_14858_gb300 import workloads as W
    mesh = mini_two_sizes()
    g = mesh.g
    fields = W.workload_fields(4)[:2]
    per_block = W.sample(mesh, fields)
    beta_blocks = W.sample(mesh, shift_fields())
    buf, bbuf = W.pack(per_block), W.pack(beta_blocks)
    Bk = bind(lib, "X2_d1", mesh, g, lib.CFD_F64)
    dev = torch.device("cuda", 0)
    nint = sum(int(n) ** 3 for n in mesh.n)
    out = torch.zeros(nint * 2, dtype=torch.float64, device=dev)
    work = torch.empty(max(lib.cfd_biased_workspace(Bk, 2, prec, 0), 256), dtype=torch.uint8, device=dev)
    lib.cfd_advect(Bk, torch.from_numpy(buf).to(dev), 2, torch.from_numpy(bbuf).to(dev), prec, 0, out, work)
    lib.cfd_sync_status(Bk)
    got = W.unpack(out.cpu().numpy(), mesh, 2, interior=True, nops=1)
    b_ = biased_of("X2_d1")
    worst = 0.0
    for q in range(2):
        want, gotq = [], []
        for b in range(mesh.nblocks):
            N = int(mesh.n[b])
            I = slice(g, g + N)
            beta = [beta_blocks[b][c][I, I, I][None, None, None] for c in range(3)]
            want.append(B.advect_uniform(per_block[b][q][None, None, None], beta, b_, mesh.dx[b], N, g, 0)[0, 0, 0])
            gotq.append(got[b][q, 0])
        wmax = max(np.abs(w).max() for w in want)
        worst = max(worst, max(np.abs(a - w).max() for a, w in zip(gotq, want)) / wmax)
    assert worst < (TOL64 if prec == 0 else TOL_TC), worst


@pytest.mark.parametrize("prec", [0, 2])
def test_biased_slab_mixed_cyclic_and_decomposed_axes(lib, torch, prec):
    """A slab of 4 x 4 x 1 blocks of 16^3: x and y decomposed (one iteration), z one block thick
    and therefore cyclic (the undecomposed periodic scheme) -- on both arithmetics."""
    from paper_2302_14858_gb300 import workloads as W
    N, g = 16, 4
    mesh = W.periodic_box_mesh(4, 4, 1, N, g)
    dx = 2 * np.pi / 64
    x = (np.arange(64) + 0.5) * dx
    z = (np.arange(16) + 0.5) * dx
    Z, Y, X = np.meshgrid(z, x, x, indexing="ij")
    fg = np.sin(3 * X - Y) * np.cos(2 * Y) + 0.3 * np.sin(X + 5 * 2 * np.pi * Z / (16 * dx))
    ext = C.ghost_fill_3d(fg, N, g)                   # (1, 4, 4, E, E, E)
    E = N + 2 * g
    buf = ext.reshape(mesh.nblocks, E, E, E).reshape(-1)
    Bk = bind(lib, "X2_d1", mesh, g, lib.CFD_F64)
    b_ = biased_of("X2_d1")
    for side in (1, -1):
        got = run_biased(lib, torch, Bk, buf, 1, lib.CFD_OP_DX | lib.CFD_OP_DY | lib.CFD_OP_DZ, side, 1, prec=prec)
        got = got.reshape(mesh.nblocks, 3, N, N, N)
        want = B.biased_uniform(ext, b_, side, (dx, dx, dx), N, g, ("x", "y"), 1)
        tol = TOL64 if prec == 0 else TOL_TC
        for i, c in enumerate(("x", "y")):
            assert rel_max(got[:, i], want[c].reshape(mesh.nblocks, N, N, N)) < tol, (side, c)
        wz = np.moveaxis(B.global_periodic(np.moveaxis(fg, 0, 0), b_, side, dx), 0, 0)
        gz = C.blocks_to_global(got[:, 2].reshape(1, 4, 4, N, N, N))
        assert rel_max(gz, wz) < tol, (side, "z")


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (2, 1e-6)])
def test_advect_long_time_matches_the_fully_discrete_prediction(lib, torch, prec, tol):
    """5000 2S steps of 2D advection (64^2 as 4 x 4 blocks of 16^2, one block thick in z; X_2 with
    one iteration, dissipation, direction 30 degrees, CFL 1/10) on the GPU equal the oracle's
    exact propagation of the same fully discrete linear system (eigen-basis form of R(dt L)^n):
    a long-time check of the upwinding, the iteration, the dissipation and the step together."""
    from oracle import timestep as T
    from paper_2302_14858_gb300 import workloads as W
    N, g, sigma, r, nsteps = 16, 4, 0.04, 4, 5000
    NM = 64
    mesh = W.periodic_box_mesh(4, 4, 1, N, g)
    E = N + 2 * g
    dx = 2 * np.pi / NM
    c = (np.cos(np.pi / 6), np.sin(np.pi / 6))
    b_ = biased_of("X2_d1")
    x = (np.arange(NM) + 0.5) * dx
    Y, X = np.meshgrid(x, x, indexing="ij")
    U0 = 0.05 * np.exp(-np.sin(2 * (X - 0.2))) * (np.exp(-1.5 * (Y - np.pi) ** 2) * (1.2 * np.sin(7 * Y) - np.cos(7 * Y))
                                                  + np.sin(2 * Y - 1.0))
    fg = np.broadcast_to(U0, (N, NM, NM)).copy()          # constant along z
    buf = C.ghost_fill_3d(fg, N, g).reshape(mesh.nblocks, E, E, E).reshape(-1)
    bb = np.empty((mesh.nblocks, 3, E, E, E))
    bb[:, 0], bb[:, 1], bb[:, 2] = -c[0], -c[1], 0.0
    Bk = bind(lib, "X2_d1", mesh, g, lib.CFD_F64)
    tu = torch.from_numpy(buf).cuda()
    tb = torch.from_numpy(bb.reshape(-1)).cuda()
    work = torch.empty(lib.cfd_advect_lsrk_workspace(Bk, 1, prec, 1), dtype=torch.uint8, device="cuda")
    coef = T.lsrk2s_rk4_float()
    dt = 0.1 * dx
    for _ in range(nsteps):
        lib.cfd_advect_lsrk_step(Bk, tu, 1, tb, dt, coef, sigma, r, prec, 1, work)
    lib.cfd_sync_status(Bk)
    got = tu.cpu().numpy().reshape(1, 4, 4, E, E, E)[:, :, :, g:g + N, g:g + N, g:g + N]
    got = C.blocks_to_global(got)                           # (z, y, x)
    Mx = T.advect_operator_1d(b_, -c[0], NM, dx, N, g, 1, sigma, r)
    My = T.advect_operator_1d(b_, -c[1], NM, dx, N, g, 1, sigma, r)
    want = T.fully_discrete_2d(Mx, My, U0, dt, nsteps)
    for zp in (0, N - 1):
        assert rel_max(got[zp], want) < tol, (zp, rel_max(got[zp], want))

