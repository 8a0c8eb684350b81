"""The device-side timeout path of the tensor-core kernel, exercised without a fault or a hang.

Every wait inside the kernel's main loop is bounded; when one runs out the kernel latches
CFD_ERR_TIMEOUT in the handle's status word, drains its own TMA copies and MMAs (with the
long default limit) and frees its tensor memory.  The test hook cfd_debug_set_wait_limit
makes the limit a few cycles, so that the first wait of every role gives up at once: nothing
hangs, the host sees the status, and the next call with the default limit is correct.
"""
import numpy as np
import pytest

from oracle import cfd as C
from paper_2302_14858_gb300 import workloads as W
from tests.helpers import OPS, desc, oracle_sch, rel_max

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2302_14858_gb300 import build
    build.build()
    from paper_2302_14858_gb300 import cfd
    return cfd


@pytest.mark.parametrize("n_iter", [0, 1])
def test_wait_limit_runs_out_then_next_call_is_correct(lib, n_iter):
    import torch
    NM, N, g = 64, 32, 4
    dx = 2 * np.pi / NM
    x = (np.arange(NM) + 0.5) * dx
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    f = W.sine_sum(W.rng(61), 8, 1, 12)
    ext = C.ghost_fill_3d(f(X, Y, Z), N, g)
    mesh = W.uniform_mesh(NM, N, g)
    s = lib.cfd_scheme_create(desc("Q13_1_d1"), desc("Q13_1_d2"))
    B = lib.cfd_blocks_bind(s, mesh.n, mesh.dx, mesh.neighbors, g, lib.CFD_F64)
    dev = torch.device("cuda", 0)
    fields = torch.from_numpy(ext.reshape(-1).copy()).to(dev)
    out = torch.empty(mesh.nblocks * 9 * N ** 3, dtype=torch.float64, device=dev)
    ws = lib.cfd_apply_workspace(B, 1, lib.CFD_OP_ALL, lib.CFD_TC_BF16_EXACT, n_iter)
    work = torch.empty(max(ws, 256), dtype=torch.uint8, device=dev)
    lib.cfd_debug_set_wait_limit(4)
    try:
        lib.cfd_apply(B, fields, 1, lib.CFD_OP_ALL, lib.CFD_TC_BF16_EXACT, n_iter, out, work)
        with pytest.raises(lib.CfdError) as e:
            lib.cfd_sync_status(B)
        assert e.value.status == lib.CFD_ERR_TIMEOUT
    finally:
        lib.cfd_debug_set_wait_limit(0)
    lib.cfd_sync_status(B)                      # cleared by the read above
    out.fill_(float("nan"))
    lib.cfd_apply(B, fields, 1, lib.CFD_OP_ALL, lib.CFD_TC_BF16_EXACT, n_iter, out, work)
    lib.cfd_sync_status(B)
    got = out.cpu().numpy().reshape(mesh.nblocks, 9, N, N, N)
    ref = C.apply_uniform(ext, oracle_sch("Q13_1_d1"), oracle_sch("Q13_1_d2"), (dx, dx, dx), N, g, OPS, n_iter)
    for i, op in enumerate(OPS):
        assert rel_max(got[:, i], ref[op].reshape(mesh.nblocks, N, N, N)) < 1e-7, op
