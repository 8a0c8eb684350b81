"""Pins of oracle.cfd: closed forms, brute force, invariants (CPU only)."""
import json
import math
import os

import numpy as np
import pytest

from oracle import cfd as C
from oracle import schemes as S
from paper_2302_14858_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
with open(os.path.join(HERE, "golden", "schemes.json")) as fh:
    SCH = json.load(fh)


def sch(name):
    e = SCH[name]
    return C.Sch(e["d"], e["a"], tuple(e["rhs"]), tuple(e["closure"]))


P1, P2 = sch("P2_d1"), sch("P2_d2")
Q1, Q2 = sch("Q13_1_d1"), sch("Q13_1_d2")
ALL = [P1, P2, Q1, Q2]
IDS = ["P1", "P2", "Q1", "Q2"]


def g_fun(x, A=0.05, Sx=1.0, N1=2, x0=0.2):
    """Eq. test_grid_conv_g with the parameters of Fig. der_01_decomp."""
    return A * np.exp(-Sx * np.sin(N1 * (x - x0)))


def g_der(x, A=0.05, Sx=1.0, N1=2, x0=0.2):
    return g_fun(x) * (-Sx * N1 * np.cos(N1 * (x - x0)))


def h_fun(x, Sx=3.0, x0=np.pi, N1=5, N2=11, phiS=3.0, c1=1.2, c2=-1.0):
    """Eq. test_grid_conv_h with the parameters of Fig. der_02_decomp (aperiodic tail is tiny)."""
    return np.exp(-Sx * (x - x0) ** 2) * (c1 * np.sin(N2 * x) + c2 * np.cos(N2 * x)) + np.sin(N1 * x - phiS)


def wavenumber(s: C.Sch, eta):
    """eta~ from Eq. fdpwerrdef for the centred tridiagonal scheme, written out."""
    M = s.M
    num = sum(s.rhs[i] * np.exp(1j * (i - M) * eta) for i in range(2 * M + 1))
    den = 1 + s.a * (np.exp(1j * eta) + np.exp(-1j * eta))
    val = num / den / (1j ** s.d)
    return val.real


# ------------------------------------------------------------------ closed forms


@pytest.mark.parametrize("s", ALL, ids=IDS)
@pytest.mark.parametrize("NM", [32, 64])
def test_global_scheme_closed_form(s, NM):
    """Circulant operator: a sine mode maps to eta~(k dx)/dx times its derivative mode."""
    dx = 2 * np.pi / NM
    x = (np.arange(NM) + 0.5) * dx
    for k, ph in ((1, 0.3), (5, 1.1), (11, 2.0), (NM // 2 - 1, 0.7)):
        f = np.sin(k * x + ph)
        et = wavenumber(s, k * dx)          # eta~^{d}
        got = C.global_periodic(f, s, dx)
        if s.d == 1:
            want = et / dx * np.cos(k * x + ph)
        else:
            want = -et / dx ** 2 * np.sin(k * x + ph)
        scale = np.abs(want).max() + 1.0 / dx ** s.d * 1e-3
        assert np.abs(got - want).max() / scale < 5e-13


def test_wavenumber_agrees_with_scheme_design():
    """The written-out eta~ equals oracle.schemes.modified_wavenumber for the printed-digit scheme family."""
    p = S.pade(1, 2)
    for eta in (0.1, 1.0, 2.5):
        assert abs(wavenumber(P1, eta) - S.modified_wavenumber(p, eta).real) < 1e-14


# ------------------------------------------------------------------ decomposition


@pytest.mark.parametrize("s", ALL, ids=IDS)
def test_iteration_converges_to_global_scheme(s):
    """Eq. iter_center_P iterated from the closure converges geometrically to the global scheme."""
    NM, N, g = 128, 16, 4
    dx = 2 * np.pi / NM
    x = (np.arange(NM) + 0.5) * dx
    f = g_fun(x) if s.d == 1 else h_fun(x)
    glob = C.global_periodic(f, s, dx)
    scale = np.abs(glob).max()
    errs = [np.abs(C.decomposed_1d(f, s, dx, N, g, i) - glob).max() / scale for i in range(7)]
    assert errs[0] < 1e-5
    for a, b in zip(errs[:5], errs[1:6]):
        assert b < a / 4, errs
    assert errs[6] < 1e-11


@pytest.mark.parametrize("s", ALL, ids=IDS)
@pytest.mark.parametrize("i", [0, 1, 2])
def test_banded_equals_embedded_operator(s, i):
    """Brute force: [i]D of Eq. iter_scheme built from dense matrices (D-bar_L, D-bar_R, G, E, Z)."""
    N, g, NS = 8, 4, 3
    dx = 0.37
    r = np.random.default_rng(7)
    f = r.standard_normal(N * NS)
    D = C.embedded_operator(s, NS, N, g, dx, i)
    F0 = C.ghost_fill_1d(f, N, g).reshape(-1)
    y = (D @ F0).reshape(NS, N + 2 * g)[:, g:g + N].reshape(-1)
    ref = C.decomposed_1d(f, s, dx, N, g, i)
    assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()


def test_ghost_fill_is_G():
    """ghost_fill_1d equals G applied to blocks whose interiors hold the data (Eq. example_G)."""
    N, g, NS = 8, 4, 4
    f = np.arange(N * NS, dtype=float) + 1
    F = np.zeros((NS, N + 2 * g))
    F[:, g:g + N] = f.reshape(NS, N)
    G = C.embedded_G(NS, N, g)
    assert np.array_equal((G @ F.reshape(-1)).reshape(NS, -1), C.ghost_fill_1d(f, N, g))


def test_exchange_ghosts_matches_periodic_fill():
    """Block-to-block copy through a 26-neighbour table equals the periodic fill of the global array."""
    N, g, NM = 4, 3, 8
    r = np.random.default_rng(3)
    fg = r.standard_normal((NM, NM, NM))
    full = C.ghost_fill_3d(fg, N, g)
    mesh = W.uniform_mesh(NM, N, g)
    nb = NM // N
    blocks = []
    for b in range(mesh.nblocks):
        bz, by, bx = b // (nb * nb), (b // nb) % nb, b % nb
        e = np.zeros((N + 2 * g,) * 3)
        e[g:g + N, g:g + N, g:g + N] = full[bz, by, bx, g:g + N, g:g + N, g:g + N]
        blocks.append(e)
    out = C.exchange_ghosts(blocks, mesh.neighbors, N, g)
    for b in range(mesh.nblocks):
        bz, by, bx = b // (nb * nb), (b // nb) % nb, b % nb
        assert np.array_equal(out[b], full[bz, by, bx])


@pytest.mark.parametrize("s", ALL, ids=IDS)
def test_polynomial_exactness(s):
    """The closed block system is exact on polynomials up to the formal order (+1 for d=2 by symmetry)."""
    N, g = 16, 4
    r = np.random.default_rng(11)
    xs = (np.arange(-g, N + g) + 0.5) * 0.1 - 0.8
    top = 6 if s.d == 1 else 7
    for deg in range(top + 1):
        p = np.polynomial.Polynomial(r.standard_normal(deg + 1))
        d = C.closed_solve(p(xs), s, 0.1, N, g)
        want = p.deriv(s.d)(xs[g:g + N])
        assert np.abs(d - want).max() <= 1e-9 * max(1.0, np.abs(want).max()), deg
    p = np.polynomial.Polynomial(r.standard_normal(top + 2))
    d = C.closed_solve(p(xs), s, 0.1, N, g)
    assert np.abs(d - p.deriv(s.d)(xs[g:g + N])).max() > 1e-8


def test_grid_convergence_sixth_order():
    """Fig. der_grid_conv: decomposed (closure only) derivatives converge at order 6."""
    N, g = 16, 4
    errs = {P1: [], Q1: [], P2: [], Q2: []}
    sizes = [64, 128, 256]
    for NM in sizes:
        dx = 2 * np.pi / NM
        x = (np.arange(NM) + 0.5) * dx
        for s in errs:
            if s.d == 1:
                f, want = g_fun(x), g_der(x)
            else:
                f = np.sin(3 * x) + 0.5 * np.cos(7 * x + 0.2)
                want = -9 * np.sin(3 * x) - 24.5 * np.cos(7 * x + 0.2)
            errs[s].append(np.abs(C.decomposed_1d(f, s, dx, N, g, 0) - want).max())
    for s, e in errs.items():
        rate = math.log2(e[1] / e[2])
        assert 5.3 < rate < 7.5, (s, e)


# ------------------------------------------------------------------ 3D


def _sep_data(NM, N, g):
    dx = 2 * np.pi / NM
    x = (np.arange(NM) + 0.5) * dx
    gx, hy, qz = g_fun(x), np.sin(2 * x + 0.4) + 0.3 * np.cos(5 * x), np.cos(3 * x + 1.0)
    fg = qz[:, None, None] * hy[None, :, None] * gx[None, None, :]
    return dx, gx, hy, qz, fg


@pytest.mark.parametrize("n_iter", [0, 1])
def test_3d_tensor_product_consistency(n_iter):
    """Separable data: each 3D op equals the 1D decomposed operators applied per factor."""
    NM, N, g = 32, 8, 4
    dx, gx, hy, qz, fg = _sep_data(NM, N, g)
    ext = C.ghost_fill_3d(fg, N, g)
    res = C.apply_uniform(ext, Q1, Q2, (dx, dx, dx), N, g, C.OPS, n_iter)
    one = {}
    for name, v in (("x", gx), ("y", hy), ("z", qz)):
        one[name] = (v, C.decomposed_1d(v, Q1, dx, N, g, n_iter), C.decomposed_1d(v, Q2, dx, N, g, n_iter))

    def outer(z, y, x):
        return z[:, None, None] * y[None, :, None] * x[None, None, :]

    want = {
        "dx": outer(qz, hy, one["x"][1]), "dy": outer(qz, one["y"][1], gx), "dz": outer(one["z"][1], hy, gx),
        "dxx": outer(qz, hy, one["x"][2]), "dyy": outer(qz, one["y"][2], gx), "dzz": outer(one["z"][2], hy, gx),
        "dxy": outer(qz, one["y"][1], one["x"][1]), "dxz": outer(one["z"][1], hy, one["x"][1]),
        "dyz": outer(one["z"][1], one["y"][1], gx),
    }
    for op in C.OPS:
        got = C.blocks_to_global(res[op])
        assert np.abs(got - want[op]).max() <= 1e-12 * np.abs(want[op]).max(), op


@pytest.mark.parametrize("n_iter", [0, 1, 2])
def test_3d_general_data_equals_line_operators(n_iter):
    """Random (non-separable) data: every 3D op equals the decomposed 1D operator applied to the
    global lines, the mixed ones as (D_i[D_j f] + D_j[D_i f]) / 2 of those line operators.  The
    separable test above pins the 3D path on tensor-product data only; a mistake that cancels
    there (ghost rows of the intermediate, the iterate a block reads across an edge) fails here."""
    NM, N, g = 32, 8, 4
    r = np.random.default_rng(77 + n_iter)
    fg = r.standard_normal((NM, NM, NM))
    dx = 2 * np.pi / NM
    res = C.apply_uniform(C.ghost_fill_3d(fg, N, g), Q1, Q2, (dx, dx, dx), N, g, C.OPS, n_iter)

    def line(f, s, axis):           # axis 0 z, 1 y, 2 x of the global array
        return np.moveaxis(C.decomposed_1d(np.moveaxis(f, axis, 0), s, dx, N, g, n_iter), 0, axis)

    ax = {"x": 2, "y": 1, "z": 0}
    want = {}
    for a in "xyz":
        want["d" + a] = line(fg, Q1, ax[a])
        want["d" + a + a] = line(fg, Q2, ax[a])
    for a, b in (("x", "y"), ("x", "z"), ("y", "z")):
        want["d" + a + b] = 0.5 * (line(want["d" + b], Q1, ax[a]) + line(want["d" + a], Q1, ax[b]))
    for op in C.OPS:
        got = C.blocks_to_global(res[op])
        assert np.abs(got - want[op]).max() <= 1e-12 * np.abs(want[op]).max(), op


def test_mixed_orders_agree_without_iteration():
    """With closures only, D_i D_j and D_j D_i are the same Kronecker operator (rounding aside)."""
    NM, N, g = 32, 8, 4
    r = np.random.default_rng(5)
    fg = r.standard_normal((NM, NM, NM))
    ext = C.ghost_fill_3d(fg, N, g)
    dx = 2 * np.pi / NM
    I = slice(g, g + N)
    data = ext[:, :, :, I, :, :]                      # z interior, y and x extended
    gy = C._axis_solve(data, 1, Q1, dx, N, g, 0, 1)   # D_y on x-extended rows
    a = C._axis_solve(gy, 2, Q1, dx, N, g, 0, 2)
    gx_ = C._axis_solve(data, 2, Q1, dx, N, g, 0, 2)
    b = C._axis_solve(gx_, 1, Q1, dx, N, g, 0, 1)
    assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()


@pytest.mark.parametrize("n_iter", [0, 1, 2])
def test_apply_block_equals_uniform_single_block(n_iter):
    """One block per axis, periodic: apply_block (closures) equals apply_uniform at n_iter=0."""
    NM, N, g = 16, 16, 4
    r = np.random.default_rng(9)
    fg = r.standard_normal((NM, NM, NM))
    ext = C.ghost_fill_3d(fg, N, g)
    dx = 2 * np.pi / NM
    a = C.apply_block(ext[0, 0, 0], Q1, Q2, (dx, dx, dx), N, g)
    b = C.apply_uniform(ext, Q1, Q2, (dx, dx, dx), N, g, C.OPS, 0)
    for op in C.OPS:
        assert np.array_equal(a[op], b[op][0, 0, 0])


# ------------------------------------------------------------------ RK4


def test_rk4_step_closed_form_per_mode():
    """Global operator: a plane wave mode is advanced by the ERK4 stability polynomial R(dt L)."""
    NM = 16
    dx = 2 * np.pi / NM
    x = (np.arange(NM) + 0.5) * dx
    k = np.array([2, 3, 1])
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    phase = k[0] * X + k[1] * Y + k[2] * Z + 0.4
    phi0, K0 = np.cos(phase), 0.7 * np.sin(phase)

    def lap(p):
        out = 0.0
        for ax in range(3):
            out = out + np.moveaxis(C.global_periodic(np.moveaxis(p, ax, 0), Q2, dx), 0, ax)
        return out

    dt = 0.25 * dx
    # one classical RK4 step written with the global Laplacian
    def rhs(p, q):
        return q, lap(p)
    k1 = rhs(phi0, K0)
    k2 = rhs(phi0 + dt / 2 * k1[0], K0 + dt / 2 * k1[1])
    k3 = rhs(phi0 + dt / 2 * k2[0], K0 + dt / 2 * k2[1])
    k4 = rhs(phi0 + dt * k3[0], K0 + dt * k3[1])
    phi1 = phi0 + dt / 6 * (k1[0] + 2 * k2[0] + 2 * k3[0] + k4[0])
    # closed form: Lambda = sum_i eta~2(k_i dx)/dx^2; state (c, s) coefficients of cos/sin
    Lam = sum(wavenumber(Q2, ki * dx) for ki in k) / dx ** 2
    Mx = np.array([[0.0, 1.0], [-Lam, 0.0]])  # acting on (phi, K) amplitudes of the same mode
    R = np.eye(2)
    term = np.eye(2)
    for n in range(1, 5):
        term = term @ (dt * Mx) / n
        R = R + term
    # phi = a cos + b sin ; K = c cos + e sin  -> evolve cos and sin parts independently
    cos_p, sin_p = np.cos(phase), np.sin(phase)
    a1 = R @ np.array([1.0, 0.0])
    b1 = R @ np.array([0.0, 0.7])
    want = (a1[0]) * cos_p + (b1[0]) * sin_p
    assert np.abs(phi1 - want).max() < 1e-13
    # and the oracle's own wave_rk4_step with the decomposed operator at n_iter=3 is close to it
    p_dec, _ = C.wave_rk4_step(phi0, K0, dt, Q2, (dx, dx, dx), 8, 4, n_iter=6)
    assert np.abs(p_dec - want).max() < 1e-9
