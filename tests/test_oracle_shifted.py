"""Pins of the shifted wave system (Eq. toyShiftWaveEqnSys) in oracle/timestep.py: the composed
right-hand side on a plane wave against the modified wavenumbers, and the end-to-end accuracy of
Sec. "Shifted wave equation" (exponential integration over 100 crossing times, N_M = 128)."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import biased as B
from oracle import cfd as C
from oracle import schemes as SC
from oracle import timestep as T
from tests.helpers import SCHEMES, oracle_sch


def _biased(name):
    e = SCHEMES[name]
    return B.Biased(e["a"], e["lo"], tuple(e["rhs"]), e["c_sup"], e["c_lo"], tuple(e["closure"]), e["kc"])


def test_shifted_wave_rhs_on_a_plane_wave():
    """Constant shift (beta^x > 0, beta^y < 0, beta^z = 0): with the iteration converged, a
    mode Re(A e^{i k.x}) of (Phi, K) is mapped by the symbols: beta^x uses the right-biased
    wavenumber, beta^y the left-biased one (Eq. biasderapproxadv with c = -beta), the
    Laplacian the second-degree scheme's, the dissipation the Kreiss-Oliger symbol."""
    NM, N, g, r, sigma, n_iter = 32, 16, 4, 4, 0.04, 12
    dx = 2 * np.pi / NM
    x = (np.arange(NM) + 0.5) * dx
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    k = (3, -2, 5)
    th = k[0] * X + k[1] * Y + k[2] * Z
    Ap, Ak = 1.0 + 0.3j, -0.2 + 0.5j
    phi, K = (Ap * np.exp(1j * th)).real, (Ak * np.exp(1j * th)).real
    bvec = (0.6, -0.4, 0.0)
    beta = [np.full_like(X, v) for v in bvec]
    b = _biased("X2_d1")
    s2 = oracle_sch("Q13_1_d2")
    fp, fk = T.shifted_wave_rhs(phi, K, beta, s2, b, (dx, dx, dx), N, g, n_iter, sigma, r)
    X2 = B.ccu_x(2, Fraction(86, 100))[0]
    q2 = SC.tuned_Q(2, 1)
    S = 0j
    lam = 0.0
    q = 0.0
    for bi, ki in zip(bvec, k):
        sch = B.mirror(X2) if bi > 0 else X2
        S += bi * 1j * SC.modified_wavenumber(sch, ki * dx) / dx
        lam += -SC.modified_wavenumber(q2, ki * dx).real / dx ** 2
        q += T.ko_symbol(r, sigma, dx, ki)
    want_p = ((Ap * S + Ak + q * Ap) * np.exp(1j * th)).real
    want_k = ((Ak * S + lam * Ap + q * Ak) * np.exp(1j * th)).real
    assert np.max(np.abs(fp - want_p)) < 1e-10 * np.max(np.abs(want_p))
    assert np.max(np.abs(fk - want_k)) < 1e-10 * np.max(np.abs(want_k))
    # taking the other bias on either axis changes the result well above that tolerance
    S_bad = bvec[0] * 1j * SC.modified_wavenumber(X2, k[0] * dx) / dx + \
        bvec[1] * 1j * SC.modified_wavenumber(B.mirror(X2), k[1] * dx) / dx
    bad = ((Ap * S_bad + Ak + q * Ap) * np.exp(1j * th)).real
    assert np.max(np.abs(bad - want_p)) > 1e-8 * np.max(np.abs(want_p))


def _initial_1d(NM):
    """Eq. ini_wav with tau = 8/100, a = 1 (a left-moving profile for beta = 1/2)."""
    dx = 2 * np.pi / NM
    x = (np.arange(NM) + 0.5) * dx
    c = (2 * np.pi * 0.08) ** -2
    s = np.sin(x / 2 - np.pi / 2)
    phi = np.exp(-c * s ** 2)
    k = phi * (-c) * s * np.cos(x / 2 - np.pi / 2)      # a d/dx phi, a = 1
    return dx, phi, k


def _ei_error(s1, s2, NM=128, beta=0.5, t=200 * np.pi):
    dx, phi, k = _initial_1d(NM)
    A1, B1 = C.cyclic_matrices(s1, NM, dx)
    A2, B2 = C.cyclic_matrices(s2, NM, dx)
    L = T.shifted_wave_1d_operator(np.linalg.solve(A1, B1), np.linalg.solve(A2, B2), beta)
    U = T.exp_integrate(L, np.concatenate([phi, k]), t)
    return np.abs(U[:NM] - phi).max()


def _explicit(d):
    r = SC.to_float_tuple(SC.explicit(d, 3).rhs_list())
    return C.Sch(d, 0.0, r, r)


def test_initial_profile_returns_after_100_crossings():
    """The continuum solution of Eq. wav2prot with beta = 1/2 and K = Phi' moves left at speed
    3/2, so at T = 200 pi the profile is back (300 pi = 150 periods): the spectral (exact)
    operators reproduce it up to a uniform offset of 9e-8 (the sampled K = Phi' has a mean of
    ~1e-10, which the exact system integrates over T)."""
    NM = 128
    dx, phi, k = _initial_1d(NM)
    n = np.fft.fftfreq(NM, 1.0 / NM)
    n1 = np.where(np.abs(n) == NM // 2, 0.0, n)         # no first derivative of the Nyquist mode
    F = np.fft.fft(np.eye(NM), axis=0)
    Fi = np.linalg.inv(F)
    D1 = (Fi @ np.diag(1j * n1) @ F).real
    D2 = (Fi @ np.diag(-n.astype(float) ** 2) @ F).real
    U = T.exp_integrate(T.shifted_wave_1d_operator(D1, D2, 0.5), np.concatenate([phi, k]), 200 * np.pi)
    err = U[:NM] - phi
    assert np.abs(err).max() < 2e-7
    assert np.abs(err - err.mean()).max() < 1e-9


def test_exponential_integration_reproduces_the_pade_error_ratio():
    """Sec. "Shifted wave equation": at N_M = 128 the implicit P^1_2 schemes reduce the maximum
    error after 100 crossing times by a factor 11.2 against the explicit E_3 (printed value);
    the oracle's circulant operators and exponential integration give 11.23.  The tuned
    Q^1_3[1] gives a reduction of about 110 here (the printed figure is 85.7; see the reading
    in the design notes): the pin only requires Q to beat P by more than a factor of 5."""
    e3 = _ei_error(_explicit(1), _explicit(2))
    p2 = _ei_error(oracle_sch("P2_d1"), oracle_sch("P2_d2"))
    q3 = _ei_error(oracle_sch("Q13_1_d1"), oracle_sch("Q13_1_d2"))
    assert abs(e3 / p2 - 11.2) < 0.1
    assert p2 / q3 > 5


def test_advection_step_advances_a_mode_by_the_stability_polynomial():
    """u_t = beta . grad u + KO with a constant shift (beta^x > 0, beta^y < 0): with the iteration
    converged a mode Re(A e^{i k.x}) is multiplied by R(dt (S + q)) per 2S step, S the upwinded
    symbol sum_i beta_i i eta~_i / dx (right-biased wavenumber where beta_i > 0, left-biased
    where beta_i < 0), q the Kreiss-Oliger symbol and R(z) = 1 + z + z^2/2 + z^3/6 + z^4/24;
    |R| <= 1 for this mode (no growth)."""
    NM, N, g, r, sigma, n_iter = 32, 16, 4, 4, 0.04, 10
    dx = 2 * np.pi / NM
    x = (np.arange(NM) + 0.5) * dx
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    k = (4, -3, 2)
    th = k[0] * X + k[1] * Y + k[2] * Z
    A = 0.7 - 0.4j
    u = (A * np.exp(1j * th)).real
    bvec = (0.5, -0.3, 0.0)
    beta = [np.full_like(X, v) for v in bvec]
    b = _biased("Q1034_1_d1")
    q34, _ = B.tuned_Q1034(1)
    dt = 0.3 * dx
    u1 = T.advect_lsrk_step(u, beta, dt, T.lsrk2s_rk4_float(), b, (dx, dx, dx), N, g, n_iter, sigma, r)
    S = 0j
    q = 0.0
    for bi, ki in zip(bvec, k):
        sch = B.mirror(q34) if bi > 0 else q34
        S += bi * 1j * SC.modified_wavenumber(sch, ki * dx) / dx
        q += T.ko_symbol(r, sigma, dx, ki)
    z = dt * (S + q)
    R = 1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24
    want = (R * A * np.exp(1j * th)).real
    assert np.max(np.abs(u1 - want)) < 1e-11 * np.max(np.abs(want))
    assert abs(R) <= 1.0
    # the step moves the mode: without the shift it is only damped by the dissipation
    u0 = T.advect_lsrk_step(u, [0 * X] * 3, dt, T.lsrk2s_rk4_float(), b, (dx, dx, dx), N, g, n_iter, sigma, r)
    assert np.max(np.abs(u0 - u1)) > 1e-2 * np.max(np.abs(u))


def test_fully_discrete_2d_equals_stepping():
    """The eigen-basis propagation of fully_discrete_2d equals 300 explicit 2S steps of the same
    semi-discrete 2D advection operator (decomposed X_2, one iteration, dissipation), and the
    upwinded operator has no growing mode (|R| <= 1)."""
    b = _biased("X2_d1")
    NM, N, g, sigma, r = 64, 16, 4, 0.04, 4
    dx = 2 * np.pi / NM
    c = (np.cos(np.pi / 6), np.sin(np.pi / 6))
    Mx = T.advect_operator_1d(b, -c[0], NM, dx, N, g, 1, sigma, r)
    My = T.advect_operator_1d(b, -c[1], NM, dx, N, g, 1, sigma, r)
    x = (np.arange(NM) + 0.5) * dx
    Y, X = np.meshgrid(x, x, indexing="ij")
    U0 = np.sin(2 * X - Y) + 0.3 * np.cos(5 * Y + 1.0)
    dt = 0.1 * dx
    U = U0.copy()
    coef = T.lsrk2s_rk4_float()
    for _ in range(300):
        U = T.lsrk2s_step((U,), dt, coef, lambda st: (st[0] @ Mx.T + My @ st[0],))[0]
    Ue = T.fully_discrete_2d(Mx, My, U0, dt, 300)
    assert np.abs(Ue - U).max() < 1e-12 * np.abs(U).max()
    lam = np.add.outer(np.linalg.eigvals(My), np.linalg.eigvals(Mx)) * dt
    R = 1 + lam + lam ** 2 / 2 + lam ** 3 / 6 + lam ** 4 / 24
    assert np.abs(R).max() <= 1 + 1e-12

