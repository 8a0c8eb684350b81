"""GPU checks of the tensor-core dense path on inputs at the edges of its number format.

The exact-slice arithmetic quantises every pencil to 39-bit fixed point relative to its
largest magnitude (a power-of-two scale per pencil) and rebuilds each output from exact
integer sums.  What that promises, and what these tests hold it to:
  - zero pencils give exact zeros;
  - the scale is per pencil, so fields near the bottom (1e-300) or top (1e300) of the
    FP64 range, and pencils whose magnitudes differ by 2^50, keep the relative accuracy;
    inside one pencil the error is bounded by ~2^-37 sum_j |D_ij| |f_j| (values below
    2^-40 of the pencil maximum contribute nothing);
  - subnormal inputs are taken as zero;
  - a NaN or an infinity in a pencil makes every output of that pencil NaN, so the
    non-finite outputs are where the FP64 banded solve has them.
References are the oracle (finite cases) and the FP64 banded path (NaN pattern).
"""
import numpy as np
import pytest

from oracle import cfd as C
from paper_2302_14858_gb300 import workloads as W
from tests.helpers import OPS, desc, oracle_sch, rel_max

pytestmark = pytest.mark.gpu

TOL64 = 1e-7
TOL32 = 1e-6


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


def run(lib, torch, B, buf, nf, prec, dtype=np.float64, mask=None, n_iter=0):
    mask = lib.CFD_OP_ALL if mask is None else mask
    dev = torch.device("cuda", 0)
    fields = torch.from_numpy(np.ascontiguousarray(buf.astype(dtype))).to(dev)
    nops = bin(mask).count("1")
    nint = sum(int(n) ** 3 for n in B.block_n)
    out = torch.full((nint * nf * nops,), 7.0, dtype=fields.dtype, device=dev)
    ws = lib.cfd_apply_workspace(B, nf, mask, prec, n_iter)
    work = torch.empty(max(ws, 256), dtype=torch.uint8, device=dev)
    lib.cfd_apply(B, fields, nf, mask, prec, n_iter, out, work)
    lib.cfd_sync_status(B)
    return out.cpu().numpy()


def setup(lib, NM, N, fg_list, dtype=np.float64):
    g = 4
    mesh = W.uniform_mesh(NM, N, g)
    E = N + 2 * g
    exts = [C.ghost_fill_3d(fg, N, g) for fg in fg_list]
    buf = np.stack([e.reshape(mesh.nblocks, E, E, E) for e in exts], axis=1).reshape(-1)
    s = lib.cfd_scheme_create(desc("Q13_1_d1"), desc("Q13_1_d2"))
    B = lib.cfd_blocks_bind(s, mesh.n, mesh.dx, mesh.neighbors, g,
                            lib.CFD_F64 if dtype == np.float64 else lib.CFD_F32)
    return mesh, exts, buf, B


def grid(NM):
    dx = 2 * np.pi / NM
    x = (np.arange(NM) + 0.5) * dx
    return dx, np.meshgrid(x, x, x, indexing="ij")


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_zero_fields_give_exact_zeros(lib, torch, dtype):
    NM, N = 64, 32
    mesh, exts, buf, B = setup(lib, NM, N, [np.zeros((NM, NM, NM))], dtype)
    for prec in (lib.CFD_TC_BF16_EXACT, lib.CFD_FP64_BANDED):
        got = run(lib, torch, B, buf, 1, prec, dtype)
        assert np.all(got == 0.0), prec


@pytest.mark.parametrize("n_iter", [0, 1])
@pytest.mark.parametrize("scale_exp", [-995, 995])
def test_fields_at_the_ends_of_the_fp64_range(lib, torch, scale_exp, n_iter):
    """sin-sum fields scaled by 2^-995 (~1e-300) and 2^995 (~1e300): same relative accuracy,
    closed and iterated (the halo passes scale each pencil by its own power of two too)."""
    NM, N = 64, 32
    dx, (Z, Y, X) = grid(NM)
    f = W.sine_sum(W.rng(41), 8, 1, 12)
    fg = np.ldexp(f(X, Y, Z), scale_exp)
    mesh, exts, buf, B = setup(lib, NM, N, [fg])
    got = run(lib, torch, B, buf, 1, lib.CFD_TC_BF16_EXACT, n_iter=n_iter).reshape(mesh.nblocks, 9, N, N, N)
    ref = C.apply_uniform(exts[0], oracle_sch("Q13_1_d1"), oracle_sch("Q13_1_d2"), (dx, dx, dx), N, 4, OPS, n_iter)
    for i, op in enumerate(OPS):
        want = ref[op].reshape(mesh.nblocks, N, N, N)
        assert np.all(np.isfinite(got[:, i])), op
        assert rel_max(got[:, i], want) < TOL64, (op, rel_max(got[:, i], want))


def test_pencil_scales_spanning_2_pow_50(lib, torch):
    """Every (z, y) line of the field carries its own power of two in [2^-25, 2^25].

    x-pencils then differ in magnitude by up to 2^50 and each keeps its relative accuracy.
    y- and z-pencils cross those scales: there every output stays within 2^-30 of
    max_j |D_ij| x max_j |f_j| of its own pencil (the a-priori bound of the slice arithmetic,
    ~2^-32 for K <= 48 terms, with slack), i.e. accuracy relative to the pencil, not the field.
    """
    NM, N, g = 64, 32, 4
    dx, (Z, Y, X) = grid(NM)
    r = W.rng(43)
    f = W.sine_sum(r, 8, 1, 12)
    p = r.integers(-25, 26, size=(NM, NM))          # exponent per (z, y) line
    fg = f(X, Y, Z) * np.ldexp(1.0, p)[:, :, None]
    mesh, exts, buf, B = setup(lib, NM, N, [fg])
    mask = lib.CFD_OP_DX | lib.CFD_OP_DY | lib.CFD_OP_DZ | lib.CFD_OP_DXX | lib.CFD_OP_DYY | lib.CFD_OP_DZZ
    ops = OPS[:6]
    got = run(lib, torch, B, buf, 1, lib.CFD_TC_BF16_EXACT, mask=mask).reshape(mesh.nblocks, 6, N, N, N)
    s1, s2 = oracle_sch("Q13_1_d1"), oracle_sch("Q13_1_d2")
    ref = C.apply_uniform(exts[0], s1, s2, (dx, dx, dx), N, g, ops, 0)
    ext = exts[0].reshape(mesh.nblocks, N + 2 * g, N + 2 * g, N + 2 * g)
    I = slice(g, g + N)
    for i, op in enumerate(ops):
        sch = s1 if len(op) == 2 else s2
        dmax = np.abs(C.embedded_D0(sch, N, g, dx))[g:g + N].max(axis=1)   # max_j |D_ij| per row
        axis = {"x": 3, "y": 2, "z": 1}[op[1]]
        sl = [slice(None), I, I, I]
        sl[axis] = slice(None)
        fmax = np.abs(ext[tuple(sl)]).max(axis=axis, keepdims=True)          # per pencil
        shape = [1, 1, 1, 1]
        shape[axis] = N
        bound = 2.0 ** -30 * dmax.reshape(shape) * fmax
        want = ref[op].reshape(mesh.nblocks, N, N, N)
        err = np.abs(got[:, i] - want)
        assert np.all(err <= bound), (op, float((err / bound).max()))
        if op in ("dx", "dxx"):
            # one scale per x-pencil: relative accuracy per pencil
            per = err.max(axis=-1) / np.abs(want).max(axis=-1)
            assert per.max() < TOL64, (op, per.max())


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_subnormal_inputs_are_taken_as_zero(lib, torch, dtype):
    """A field of subnormal values gives exact zeros on the tensor cores (the FP64 banded
    solve resolves it); a subnormal block inside a normal field leaves the field's relative
    error against the oracle unchanged."""
    NM, N, g = 64, 32, 4
    dx, (Z, Y, X) = grid(NM)
    base = W.sine_sum(W.rng(47), 8, 1, 12)(X, Y, Z).astype(dtype).astype(np.float64)
    sub = np.finfo(dtype).tiny / 4                            # a subnormal of the field dtype
    all_sub = np.where(np.abs(base) > 0.1, np.sign(base) * sub, 0.0)
    mesh, exts, buf, B = setup(lib, NM, N, [all_sub], dtype)
    assert np.all(run(lib, torch, B, buf, 1, lib.CFD_TC_BF16_EXACT, dtype) == 0.0)
    if dtype == np.float64:
        assert np.any(run(lib, torch, B, buf, 1, lib.CFD_FP64_BANDED, dtype) != 0.0)
    mixed = base.copy()
    mixed[:N, :N, :N] = all_sub[:N, :N, :N]                   # block 0 subnormal
    mesh, exts, buf, B = setup(lib, NM, N, [mixed], dtype)
    got = run(lib, torch, B, buf, 1, lib.CFD_TC_BF16_EXACT, dtype).reshape(mesh.nblocks, 9, N, N, N)
    ref = C.apply_uniform(exts[0], oracle_sch("Q13_1_d1"), oracle_sch("Q13_1_d2"), (dx, dx, dx), N, g, OPS, 0)
    tol = TOL64 if dtype == np.float64 else TOL32
    for i, op in enumerate(OPS):
        assert rel_max(got[:, i], ref[op].reshape(mesh.nblocks, N, N, N)) < tol, op


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_nan_and_inf_propagate_like_the_banded_solve(lib, torch, dtype):
    NM, N, g = 64, 32, 4
    dx, (Z, Y, X) = grid(NM)
    fg = W.sine_sum(W.rng(53), 8, 1, 12)(X, Y, Z)
    fg[5, 7, 9] = np.nan                                      # block 0
    fg[40, 50, 20] = np.inf                                   # another block
    fg[20, 10, 60] = -np.inf
    mesh, exts, buf, B = setup(lib, NM, N, [fg], dtype)
    tc = run(lib, torch, B, buf, 1, lib.CFD_TC_BF16_EXACT, dtype).reshape(mesh.nblocks, 9, -1)
    bd = run(lib, torch, B, buf, 1, lib.CFD_FP64_BANDED, dtype).reshape(mesh.nblocks, 9, -1)
    with np.errstate(invalid="ignore", over="ignore"):
        ref = C.apply_uniform(exts[0], oracle_sch("Q13_1_d1"), oracle_sch("Q13_1_d2"), (dx, dx, dx), N, g, OPS, 0)
    tol = TOL64 if dtype == np.float64 else TOL32
    for i, op in enumerate(OPS):
        nf_tc, nf_bd = ~np.isfinite(tc[:, i]), ~np.isfinite(bd[:, i])
        assert nf_tc.any(), op
        assert np.array_equal(nf_tc, nf_bd), (op, int(nf_tc.sum()), int(nf_bd.sum()))
        assert np.all(np.isnan(tc[:, i][nf_tc])), op            # the tensor-core path writes NaN
        # the finite outputs keep their accuracy
        want = ref[op].reshape(mesh.nblocks, -1)
        fin = ~nf_tc & np.isfinite(want)
        den = np.abs(want[fin]).max()
        assert np.abs(tc[:, i][fin] - want[fin]).max() / den < tol, op
