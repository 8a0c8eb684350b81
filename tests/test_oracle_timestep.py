"""Pins of oracle/timestep.py: Kreiss-Oliger dissipation (Eq. dissdef, Tab. diss_scheme) and the
two-register (2S) Runge-Kutta recurrence with its 4-stage 4th-order coefficients."""
import json
import os
from fractions import Fraction

import mpmath as mp
import numpy as np
import pytest

from oracle import cfd as C
from oracle import schemes as SC
from oracle import timestep as T
from tests.helpers import oracle_sch, rel_max

HERE = os.path.dirname(os.path.abspath(__file__))
TAB = json.load(open(os.path.join(HERE, "golden", "paper_tables.json")))["diss_scheme"]


@pytest.mark.parametrize("r", [2, 3, 4, 5, 6])
def test_ko_stencil_is_the_printed_E_r(r):
    """dx^{2r} (D_+)^r (D_-)^r on a unit impulse is the row (2r)E_r of Tab. diss_scheme."""
    n = 4 * r + 8
    f = np.zeros(n)
    f[n // 2] = 1.0
    dx = 1.0
    # undo the prefactor of Eq. dissdef: Q = -((-1)^r / 2^{2r}) sigma dx^{2r-1} D
    q = T.ko_1d(f, 0, r, 1.0, dx)
    D = q / (-((-1) ** r) / 2.0 ** (2 * r))
    got = [round(v) for v in D[n // 2 - r:n // 2 + r + 1]]
    assert np.allclose(D[n // 2 - r:n // 2 + r + 1], got)
    assert got == TAB["rows"][str(r)]["stencil"]


@pytest.mark.parametrize("r", [2, 3, 4, 5, 6])
def test_printed_E_r_is_the_explicit_degree_2r_scheme(r):
    """The oracle's explicit scheme of degree 2r on 2r+1 points reproduces the printed stencil and
    the printed leading terms of its wavenumber error (Tab. diss_scheme)."""
    s = SC.solve_exact(SC.Ansatz(2 * r, (0, 0), ((0, r, r),)), 2)   # degree 2r, order dx^2
    row = TAB["rows"][str(r)]
    assert [Fraction(v) for v in s.rhs_list()] == [Fraction(v) for v in row["stencil"]]
    eps = SC.eps_series(s, 6)
    assert eps[2] == Fraction(*row["eps2"])
    assert eps[4] == Fraction(*row["eps4"])


@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_ko_symbol_closed_form(r):
    """Q^{(2r)} acts on exp(ikx) by -(sigma/dx) sin^{2r}(k dx/2): dissipative, vanishing at k = 0."""
    n, sigma = 64, 0.04
    dx = 2 * np.pi / n
    x = np.arange(n) * dx
    for k in (1, 5, 17, 31):
        for f in (np.sin(k * x + 0.3), np.cos(k * x - 1.1)):
            q = T.ko_1d(f, 0, r, sigma, dx)
            want = T.ko_symbol(r, sigma, dx, k) * f
            assert np.max(np.abs(q - want)) < 1e-12 * max(1.0, np.max(np.abs(want)))
        assert T.ko_symbol(r, sigma, dx, k) < 0
    assert T.ko_symbol(r, sigma, dx, 0) == 0


def test_ko_sums_the_three_directions():
    n, sigma, r = 16, 0.02, 4
    dx3 = (2 * np.pi / n, 2 * np.pi / n * 1.5, 2 * np.pi / n * 0.75)
    rng = np.random.default_rng(5)
    f = rng.standard_normal((n, n, n))
    total = T.ko_dissipation(f, r, sigma, dx3)
    # one direction at a time through a transposed call
    parts = [T.ko_1d(f, 2, r, sigma, dx3[0]), np.moveaxis(T.ko_1d(np.moveaxis(f, 1, 2), 2, r, sigma, dx3[1]), 2, 1),
             np.moveaxis(T.ko_1d(np.moveaxis(f, 0, 2), 2, r, sigma, dx3[2]), 2, 0)]
    assert np.max(np.abs(total - sum(parts))) < 1e-12 * np.max(np.abs(total))


def test_lsrk2s_coefficients_are_fourth_order():
    co = T.lsrk2s_rk4()
    with mp.workdps(50):
        A, b, c, u = T.lsrk2s_butcher(co)
        assert max(abs(v) for v in T.order4_conditions(A, b, c)) < mp.mpf(10) ** -40
        assert max(abs(v - 1) for v in u) < mp.mpf(10) ** -40
        R = T.stability_polynomial(A, b)
        want = [1, 1, mp.mpf(1) / 2, mp.mpf(1) / 6, mp.mpf(1) / 24]
        assert max(abs(a - w) for a, w in zip(R, want)) < mp.mpf(10) ** -40
        # explicit and of 4 stages: A strictly lower triangular
        assert all(abs(A[i][j]) < mp.mpf(10) ** -45 for i in range(4) for j in range(i, 4))
    # a deliberate slip in one coefficient breaks fourth order
    g1, g2, beta, delta = co
    bad = (g1, g2, [beta[0], beta[1] * (1 + mp.mpf("1e-6")), beta[2], beta[3]], delta)
    A, b, c, _ = T.lsrk2s_butcher(bad)
    assert max(abs(v) for v in T.order4_conditions(A, b, c)) > mp.mpf(10) ** -9


def test_lsrk2s_equals_erk4_on_the_wave_system():
    """Linear autonomous system: every 4-stage 4th-order method gives the same step."""
    NM, N, g = 16, 8, 4
    s2 = oracle_sch("Q13_1_d2")
    dx = 2 * np.pi / NM
    x = (np.arange(NM) + 0.5) * dx
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    phi = np.sin(2 * X + Y - Z) + 0.3 * np.cos(X - 3 * Z)
    K = np.cos(X + 2 * Y)
    dt = 0.25 * dx
    coef = T.lsrk2s_rk4_float()
    rhs = lambda st: C.wave_rhs(st[0], st[1], s2, (dx, dx, dx), N, g, 1)
    p2, k2 = T.lsrk2s_step((phi, K), dt, coef, rhs)
    p4, k4 = C.wave_rk4_step(phi, K, dt, s2, (dx, dx, dx), N, g, 1)
    assert rel_max(p2, p4) < 1e-13
    assert rel_max(k2, k4) < 1e-13


def test_lsrk2s_with_ko_advances_a_mode_by_the_stability_polynomial():
    """Undecomposed periodic operator (circulant) plus KO: the mode (Phi, K) of wave vector k is
    advanced by R(dt M), M = [[q, 1], [lambda, q]], lambda = -sum_i eta2(k_i dx)^2 / dx^2 ... with
    eta2 the second-degree scheme's modified wavenumber factor and q the summed KO symbol."""
    n, r, sigma = 32, 4, 0.04
    s2 = oracle_sch("Q13_1_d2")
    dx = 2 * np.pi / n
    x = np.arange(n) * dx
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    k = (3, -2, 5)
    arg = k[0] * X + k[1] * Y + k[2] * Z
    phi0, K0 = np.cos(arg), 0.5 * np.sin(arg)

    def lap(f):
        out = np.zeros_like(f)
        for ax in range(3):
            out += np.moveaxis(C.global_periodic(np.moveaxis(f, ax, 0), s2, dx), 0, ax)
        return out

    def rhs(st):
        p, q = st
        return q + T.ko_dissipation(p, r, sigma, (dx, dx, dx)), lap(p) + T.ko_dissipation(q, r, sigma, (dx, dx, dx))

    dt = 0.25 * dx
    p1, k1 = T.lsrk2s_step((phi0, K0), dt, T.lsrk2s_rk4_float(), rhs)
    # eigenvalue of the cyclic second-derivative operator on the mode, per axis, read off the operator
    lam = 0.0
    for kk in k:
        f1 = np.cos(kk * x)
        lam += (C.global_periodic(f1[:, None], s2, dx)[:, 0] / f1)[0]
    qk = sum(T.ko_symbol(r, sigma, dx, kk) for kk in k)
    M = np.array([[qk, 1.0], [lam, qk]]) * dt
    R = np.eye(2) + M + M @ M / 2 + M @ M @ M / 6 + M @ M @ M @ M / 24
    # cos and sin parts evolve with the same real 2x2 map
    cpart = np.array([1.0, 0.0])      # (Phi, K) coefficients of cos(arg)
    spart = np.array([0.0, 0.5])      # (Phi, K) coefficients of sin(arg)
    ca, sa = R @ cpart, R @ spart
    want_p = ca[0] * np.cos(arg) + sa[0] * np.sin(arg)
    want_k = ca[1] * np.cos(arg) + sa[1] * np.sin(arg)
    assert rel_max(p1, want_p) < 1e-12
    assert rel_max(k1, want_k) < 1e-12
    # the dissipation is visible: the same step without it differs
    p0, _ = T.lsrk2s_step((phi0, K0), dt, T.lsrk2s_rk4_float(), lambda st: (st[1], lap(st[0])))
    assert rel_max(p0, p1) > 1e-9
