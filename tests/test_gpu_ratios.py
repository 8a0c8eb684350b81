"""The paper's accuracy ratios (Secs. "Shifted wave equation", "Two dimensional advection") from
the GPU's own operators.

The ratios compare the maximum error after T = 200 pi of the semi-discrete evolution, solved by
exponential integration (Eqs. exp_integ_adv2 and its shifted-wave counterpart), for the
implicit schemes P^1_2 and Q^1_3[eta_c = 1] against the explicit E_3.  Resolving errors of
1e-7 by time stepping over 100 crossing times would need ~10^6 RK4 steps, so the check takes
the discrete operators the GPU applies: cfd_apply on unit-vector fields along x (the fields are
constant in y and z) returns the columns of the decomposed operator [1]D (N_B = 16, N_g = 4,
one hybrid iteration -- the paper's domain-decomposed runs), from the FP64 banded solves.  The
exponential integration of those operators is analysis on the host.  (The tensor-core operators
agree with them to ~1e-11 relative, but over 100 crossing times the 1+1 system integrates any
nonzero D2 . 1 twice: the constant mode of K grows linearly and Phi quadratically in t, so
operator errors at that level reach the 1e-6 scale of the errors being compared, the same
mechanism that makes the printed 8-digit coefficients unusable there.)

Printed: 1+1 shifted wave at N_M = 128: 11.2 (P), 85.7 (Q); 2D advection at 192^2: 13.6 (P),
65.9 (Q).  This library and its oracle give 11.2 and ~110 (1+1), 14.6 and ~145 (2D): the P
ratios agree (within 0.1 and 7 %), the Q ratios do not (see the design notes for the readings
tried).  The test asserts the P ratios against the paper and every ratio against the same
computation on the oracle's operators.
"""
import math

import numpy as np
import pytest

from oracle import cfd as C
from oracle import schemes as SC
from oracle import timestep as T
from paper_2302_14858_gb300 import workloads as W
from tests.helpers import SCHEMES, oracle_sch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2302_14858_gb300 import build
    build.build()
    from paper_2302_14858_gb300 import cfd
    return cfd


def lib_desc(name, d):
    """Library scheme descriptors: the tuned / Pade schemes with their closures, and the explicit
    E_3 with its own stencil as closure (an explicit scheme needs no closure: its stencil reads the
    ghosts, so decomposition leaves it unchanged, Sec. "Two dimensional advection")."""
    if name == "E3":
        r = [float(v) for v in SC.to_float_tuple(SC.explicit(d, 3).rhs_list())]
        return {"deriv": d, "order": 6, "a": 0.0, "rhs": r, "closure": [0.0] + r + [0.0]}  # half-width 4
    e = SCHEMES[f"{name}_d{d}"]
    return {"deriv": d, "order": e["order"], "a": e["a"], "rhs": e["rhs"], "closure": e["closure"]}


def oracle_scheme(name, d):
    if name == "E3":
        r = SC.to_float_tuple(SC.explicit(d, 3).rhs_list())
        return C.Sch(d, 0.0, r, r)
    return oracle_sch(f"{name}_d{d}")


def gpu_operators(lib, name, NM, prec, n_iter=1, N=16, g=4, degrees=(1, 2)):
    """Columns of the decomposed d_x (and d_xx) operators the GPU applies on NM points along x."""
    import torch
    mesh = W.periodic_box_mesh(NM // N, 1, 1, N, g)
    d1 = lib_desc(name, 1) if 1 in degrees else None
    d2 = lib_desc(name, 2) if 2 in degrees else None
    s = lib.cfd_scheme_create(d1, d2)
    B = lib.cfd_blocks_bind(s, mesh.n, mesh.dx, mesh.neighbors, g, lib.CFD_F64)
    E = N + 2 * g
    nf = NM
    buf = np.zeros((mesh.nblocks, nf, E, E, E))
    for q in range(NM):                          # field q: the unit vector at global x index q
        buf[q // N, q, :, :, g + q % N] = 1.0
    dev = torch.device("cuda", 0)
    fields = torch.from_numpy(buf.reshape(-1)).to(dev)
    lib.cfd_exchange_ghosts(B, fields, nf)
    mask = (lib.CFD_OP_DX if 1 in degrees else 0) | (lib.CFD_OP_DXX if 2 in degrees else 0)
    nops = bin(mask).count("1")
    out = torch.empty(mesh.nblocks * nf * nops * N ** 3, dtype=torch.float64, device=dev)
    ws = lib.cfd_apply_workspace(B, nf, mask, prec, n_iter)
    work = torch.empty(max(ws, 256), dtype=torch.uint8, device=dev)
    lib.cfd_apply(B, fields, nf, mask, prec, n_iter, out, work)
    lib.cfd_sync_status(B)
    o = out.cpu().numpy().reshape(mesh.nblocks, nf, nops, N, N, N)[:, :, :, 0, 0, :]   # (block, field, op, x)
    ops = np.transpose(o, (2, 0, 3, 1)).reshape(nops, NM, NM)   # op, global x (row), field = column
    return list(ops)


def oracle_operators(name, NM, n_iter=1, N=16, g=4, degrees=(1, 2)):
    dx = 2 * np.pi / NM
    return [C.decomposed_1d(np.eye(NM), oracle_scheme(name, d), dx, N, g, n_iter) for d in degrees]


def wave_error(D1, D2, NM, beta=0.5, t=200 * np.pi):
    """Eq. ini_wav (tau = 8/100, a = 1) evolved by exp(t L), L = [[beta D1, I], [D2, beta D1]]; the
    maximum error of Phi against the initial profile after 100 crossing times."""
    dx = 2 * np.pi / NM
    x = (np.arange(NM) + 0.5) * dx
    c = (2 * np.pi * 0.08) ** -2
    sn = np.sin(x / 2 - np.pi / 2)
    phi = np.exp(-c * sn ** 2)
    k = phi * (-c) * sn * np.cos(x / 2 - np.pi / 2)
    U = T.exp_integrate(T.shifted_wave_1d_operator(D1, D2, beta), np.concatenate([phi, k]), t)
    return float(np.abs(U[:NM] - phi).max())


def advection_error(D, NM, angle, t=200 * np.pi):
    """Eq. exp_integ_adv2 for the profile g(x) h(y) of Sec. "Two dimensional advection" moving in
    direction `angle`; the maximum error against the exactly translated profile."""
    import scipy.linalg as sl
    dx = 2 * np.pi / NM
    x = (np.arange(NM) + 0.5) * dx
    X, Y = np.meshgrid(x, x, indexing="ij")

    def prof(px, py):
        gx = 0.05 * np.exp(-1.0 * np.sin(2 * (px - 0.2)))
        hy = np.exp(-1.5 * (py - math.pi) ** 2) * (1.2 * np.sin(7 * py) - np.cos(7 * py)) + np.sin(2 * py - 1.0)
        return gx * hy

    cx, cy = math.cos(angle), math.sin(angle)
    U = sl.expm(-t * cx * D) @ prof(X, Y) @ sl.expm(-t * cy * D).T
    exact = prof(np.mod(X - t * cx, 2 * np.pi), np.mod(Y - t * cy, 2 * np.pi))
    return float(np.abs(U - exact).max())


def test_shifted_wave_ratios_from_gpu_operators(lib):
    NM = 128
    p, prec = lib.CFD_FP64_BANDED, "banded"
    err, err_o = {}, {}
    for name in ("E3", "P2", "Q13_1"):
        D1, D2 = gpu_operators(lib, name, NM, p)
        O1, O2 = oracle_operators(name, NM)
        # the GPU's operators are the oracle's
        assert np.abs(D1 - O1).max() < 1e-12 * np.abs(O1).max()
        assert np.abs(D2 - O2).max() < 1e-12 * np.abs(O2).max()
        err[name] = wave_error(D1, D2, NM)
        err_o[name] = wave_error(O1, O2, NM)
    rp, rq = err["E3"] / err["P2"], err["E3"] / err["Q13_1"]
    print(f"1+1 shifted wave, N_M = 128, N_B = 16, one iteration ({prec}): E3/P2 = {rp:.2f} (printed 11.2), "
          f"E3/Q13_1 = {rq:.1f} (printed 85.7)")
    assert abs(rp - 11.2) < 0.15
    assert abs(rp - err_o["E3"] / err_o["P2"]) < 1e-3 * rp
    assert abs(rq - err_o["E3"] / err_o["Q13_1"]) < 1e-2 * rq


def test_advection_2d_ratios_from_gpu_operators(lib):
    NM = 192
    angles = [math.radians(a) for a in (0.0, 30.0, 60.0, 90.0)]
    err, err_o = {}, {}
    for name in ("E3", "P2", "Q13_1"):
        (D,) = gpu_operators(lib, name, NM, lib.CFD_FP64_BANDED, degrees=(1,))
        (O,) = oracle_operators(name, NM, degrees=(1,))
        assert np.abs(D - O).max() < 1e-12 * np.abs(O).max()
        err[name] = max(advection_error(D, NM, a) for a in angles)
        err_o[name] = max(advection_error(O, NM, a) for a in angles)
    rp, rq = err["E3"] / err["P2"], err["E3"] / err["Q13_1"]
    print(f"2D advection, 192^2, N_B = 16, one iteration: E3/P2 = {rp:.2f} (printed 13.6), "
          f"E3/Q13_1 = {rq:.1f} (printed 65.9)")
    assert abs(rp - 13.6) < 0.1 * 13.6
    assert abs(rp - err_o["E3"] / err_o["P2"]) < 1e-3 * rp
    assert abs(rq - err_o["E3"] / err_o["Q13_1"]) < 1e-2 * rq
