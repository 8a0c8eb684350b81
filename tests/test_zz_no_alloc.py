"""The allocation-free entry point cfd_apply_static, checked against the oracle and cfd_apply.

Callers that cannot allocate device memory when they apply the operators
(their host code owns all device memory, or their loop must not allocate or
synchronise) use cfd_apply_static, whose scratch is a static 64 MiB device
array inside the library.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from oracle import cfd as C
from paper_2302_14858_gb300 import workloads as W
from tests.helpers import OPS, desc, oracle_sch, rel_max

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2302_14858_gb300 import build
    build.build()
    from paper_2302_14858_gb300 import cfd
    return cfd, torch


def _fields(NM, N, g, seeds):
    dx = 2 * np.pi / NM
    x = (np.arange(NM) + 0.5) * dx
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    mesh = W.uniform_mesh(NM, N, g)
    E = N + 2 * g
    exts = []
    for s in seeds:
        r = W.rng(s)
        f = W.Sum([W.sine_sum(r, 8, 1, 12), W.gaussian(r, 0.1)])
        exts.append(C.ghost_fill_3d(f(X, Y, Z), N, g))
    flat = np.stack([e.reshape(mesh.nblocks, E, E, E) for e in exts], axis=1).reshape(-1)
    return mesh, flat, exts


def test_static_scratch_matches_workspace_path_twice(env):
    cfd, torch = env
    NM, N, g, nf = 64, 16, 4, 2
    dx = 2 * np.pi / NM
    mesh, buf1, ext1 = _fields(NM, N, g, (501, 502))
    _, buf2, ext2 = _fields(NM, N, g, (503, 504))
    s = cfd.cfd_scheme_create(desc("Q13_1_d1"), desc("Q13_1_d2"))
    B = cfd.cfd_blocks_bind(s, mesh.n, mesh.dx, mesh.neighbors, g, cfd.CFD_F64)
    nout = mesh.nblocks * nf * 9 * N ** 3
    ws = cfd.cfd_apply_workspace(B, nf, cfd.CFD_OP_ALL, cfd.CFD_FP64_BANDED, 0)
    work = torch.empty(ws, dtype=torch.uint8, device="cuda")
    s1, s2 = oracle_sch("Q13_1_d1"), oracle_sch("Q13_1_d2")
    for buf, exts in ((buf1, ext1), (buf2, ext2)):     # two calls in a row, different data
        f = torch.from_numpy(buf).cuda()
        ref = torch.empty(nout, dtype=torch.float64, device="cuda")
        got = torch.full((nout,), float("nan"), dtype=torch.float64, device="cuda")
        cfd.cfd_apply(B, f, nf, cfd.CFD_OP_ALL, cfd.CFD_FP64_BANDED, 0, ref, work)
        cfd.cfd_apply_static(B, f, nf, cfd.CFD_OP_ALL, got)
        cfd.cfd_sync_status(B)
        r = ref.cpu().numpy().reshape(mesh.nblocks, nf, 9, -1)
        o = got.cpu().numpy().reshape(mesh.nblocks, nf, 9, -1)
        assert np.isfinite(o).all()
        for q in range(nf):
            want = C.apply_uniform(exts[q], s1, s2, (dx, dx, dx), N, g, OPS, 0)
            for i, op in enumerate(OPS):
                assert rel_max(o[:, q, i], want[op].reshape(mesh.nblocks, -1)) < TOL64, (q, op)
                assert rel_max(o[:, q, i], r[:, q, i]) < TOL64


def test_static_scratch_rejects_oversized_request(env):
    cfd, torch = env
    NM, N, g, nf = 128, 16, 4, 3         # mixed-op scratch: 3 x 512 x 24*16*16 doubles = 75.5 MB > 64 MiB
    mesh = W.uniform_mesh(NM, N, g)
    E = N + 2 * g
    s = cfd.cfd_scheme_create(desc("Q13_1_d1"), desc("Q13_1_d2"))
    B = cfd.cfd_blocks_bind(s, mesh.n, mesh.dx, mesh.neighbors, g, cfd.CFD_F64)
    f = torch.zeros(mesh.nblocks * nf * E ** 3, dtype=torch.float64, device="cuda")
    out = torch.zeros(mesh.nblocks * nf * 9 * N ** 3, dtype=torch.float64, device="cuda")
    with pytest.raises(cfd.CfdError) as e:
        cfd.cfd_apply_static(B, f, nf, cfd.CFD_OP_ALL, out)
    assert e.value.status == cfd.CFD_ERR_ARG
    assert "static array" in str(e.value)
    # single-axis ops need no scratch, so the same size is accepted
    cfd.cfd_apply_static(B, f, nf, cfd.CFD_OP_DX | cfd.CFD_OP_DZZ, out)
    cfd.cfd_sync_status(B)
