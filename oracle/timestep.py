"""Time stepping around the derivative operators: Kreiss-Oliger dissipation and a
low-storage (two-register) Runge-Kutta method.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* Kreiss-Oliger dissipation, Eq. dissdef (Sec. "Two dimensional advection"):
      Q^{(2r)} = -((-1)^r / 2^{2r}) sigma dx^{2r-1} (D_+)^r (D_-)^r,
      D_+- f_i = +-(f_{i+-1} - f_i) / dx,
  added to the right-hand side of every field component in every direction.  Here it
  is applied literally (r forward, r backward one-sided differences) on periodic
  global arrays.  (D_+)^r (D_-)^r is the stencil of (2r)E_r in Tab. diss_scheme.
* The low-storage method: the paper's host code evolves with the 4-stage, 4th-order
  RK4()4[2S] scheme of the cited Ketcheson (2010) paper (Sec. "Z4c: system
  description") but prints no coefficients.  This module states the two-register 2S
  recurrence (per stage i = 1..m, with S1 the state and S2 = 0 on entry)
      S2 <- S2 + delta_i S1
      S1 <- gamma1_i S1 + gamma2_i S2 + beta_i dt F(S1_old)
  (F evaluated at S1 before the stage updates it), maps it to its Butcher tableau,
  and finds one 4-stage 4th-order member by solving the order conditions in mpmath
  (with delta_1 = delta_4 = 1, gamma1_1 = 0, gamma2_1 = 1 the solutions still form a
  curve; minimum-norm Newton steps from a fixed start pick one point).  On a linear
  autonomous system every 4-stage 4th-order method advances a mode by the same
  polynomial 1 + z + z^2/2 + z^3/6 + z^4/24, so this member and classical ERK4
  agree there up to rounding.
* The shifted wave system (Eq. toyShiftWaveEqnSys, flat background gamma^{ij} =
  delta^{ij}): F_Phi = beta^j d_j Phi + K, F_K = beta^j d_j K + gamma^{ij} d_i d_j Phi, with
  the advective terms upwinded by the biased schemes (Eq. biasderapproxadv with c -> beta,
  Sec. "Shifted wave equation"), plus the Kreiss-Oliger terms.
* ``shifted_wave_1d_operator``: the single-domain semi-discrete operator L of Eq.
  sd_wave_ops in 1+1 dimensions (constant beta, centred circulant D^{(1)}, D^{(2)}), and
  ``exp_integrate`` its exponential integration (the paper evaluates matrix exponentials
  by the scaling-and-squaring method of its citation; scipy's expm implements that method).
"""
from __future__ import annotations

import functools
from typing import Callable, List, Sequence, Tuple

import mpmath as mp
import numpy as np

# ---------------------------------------------------------------------------
# Kreiss-Oliger dissipation (Eq. dissdef)
# ---------------------------------------------------------------------------


def ko_1d(f: np.ndarray, axis: int, r: int, sigma: float, dx: float) -> np.ndarray:
    """Q^{(2r)} of Eq. dissdef along ``axis`` of a periodic array: r backward differences
    D_-, then r forward differences D_+, times -((-1)^r / 2^{2r}) sigma dx^{2r-1}."""
    h = f
    for _ in range(r):
        h = (h - np.roll(h, 1, axis=axis)) / dx        # D_- f_i = -(f_{i-1} - f_i)/dx
    for _ in range(r):
        h = (np.roll(h, -1, axis=axis) - h) / dx       # D_+ f_i = (f_{i+1} - f_i)/dx
    return -((-1) ** r / 2.0 ** (2 * r)) * sigma * dx ** (2 * r - 1) * h


def ko_dissipation(f: np.ndarray, r: int, sigma: float, dx3: Sequence[float]) -> np.ndarray:
    """Sum of Q^{(2r)} over the three directions of a periodic (z, y, x) array;
    ``dx3`` = (dx_x, dx_y, dx_z)."""
    return (ko_1d(f, 2, r, sigma, dx3[0]) + ko_1d(f, 1, r, sigma, dx3[1])
            + ko_1d(f, 0, r, sigma, dx3[2]))


def ko_symbol(r: int, sigma: float, dx: float, k: float) -> float:
    """Eigenvalue of Q^{(2r)} on exp(i k x): (D_+ D_-) has -4 sin^2(k dx/2)/dx^2, hence
    -(sigma/dx) sin^{2r}(k dx / 2)."""
    return -(sigma / dx) * np.sin(k * dx / 2.0) ** (2 * r)


# ---------------------------------------------------------------------------
# Two-register (2S) low-storage Runge-Kutta
# ---------------------------------------------------------------------------


def lsrk2s_step(state: Tuple[np.ndarray, ...], dt: float, coef, rhs: Callable) -> Tuple[np.ndarray, ...]:
    """One step of the 2S recurrence for a tuple of arrays; ``coef`` = (gamma1, gamma2,
    beta, delta), each of length m; ``rhs(state) -> tuple`` is F."""
    gamma1, gamma2, beta, delta = coef
    S1 = tuple(np.array(a, dtype=np.float64) for a in state)
    S2 = tuple(np.zeros_like(a) for a in S1)
    for i in range(len(beta)):
        F = rhs(S1)
        S2 = tuple(s2 + delta[i] * s1 for s1, s2 in zip(S1, S2))
        S1 = tuple(gamma1[i] * s1 + gamma2[i] * s2 + beta[i] * dt * fi for s1, s2, fi in zip(S1, S2, F))
    return S1


def lsrk2s_butcher(coef):
    """Butcher tableau (A, b, c) of the 2S recurrence, and the coefficients of the state u_n
    in every stage input and in the result (all must be 1 for a consistent method).

    S1 and S2 are tracked as linear combinations of [u_n, dt k_1, ..., dt k_m]."""
    gamma1, gamma2, beta, delta = coef
    m = len(beta)
    one = beta[0] * 0 + 1
    S1 = [one] + [one * 0] * m
    S2 = [one * 0] * (m + 1)
    A, ucoef = [], []
    for i in range(m):
        A.append(S1[1:])
        ucoef.append(S1[0])
        S2 = [s2 + delta[i] * s1 for s1, s2 in zip(S1, S2)]
        S1 = [gamma1[i] * s1 + gamma2[i] * s2 for s1, s2 in zip(S1, S2)]
        S1[1 + i] = S1[1 + i] + beta[i]
    ucoef.append(S1[0])
    b = S1[1:]
    c = [sum(row) for row in A]
    return A, b, c, ucoef


def order4_conditions(A, b, c) -> List[object]:
    """The eight order conditions of an explicit RK method up to order 4 (residuals)."""
    m = len(b)
    Ac = [sum(A[i][j] * c[j] for j in range(m)) for i in range(m)]
    Ac2 = [sum(A[i][j] * c[j] ** 2 for j in range(m)) for i in range(m)]
    AAc = [sum(A[i][j] * Ac[j] for j in range(m)) for i in range(m)]
    return [sum(b) - 1,
            sum(b[i] * c[i] for i in range(m)) - mp.mpf(1) / 2,
            sum(b[i] * c[i] ** 2 for i in range(m)) - mp.mpf(1) / 3,
            sum(b[i] * Ac[i] for i in range(m)) - mp.mpf(1) / 6,
            sum(b[i] * c[i] ** 3 for i in range(m)) - mp.mpf(1) / 4,
            sum(b[i] * c[i] * Ac[i] for i in range(m)) - mp.mpf(1) / 8,
            sum(b[i] * Ac2[i] for i in range(m)) - mp.mpf(1) / 12,
            sum(b[i] * AAc[i] for i in range(m)) - mp.mpf(1) / 24]


def stability_polynomial(A, b) -> List[object]:
    """Coefficients of R(z) = 1 + z b^T (I - zA)^{-1} 1 (A strictly lower triangular)."""
    m = len(b)
    # (I - zA)^{-1} 1 = sum_k z^k A^k 1
    coeffs = [mp.mpf(1)]
    v = [mp.mpf(1)] * m
    for k in range(m):
        coeffs.append(sum(b[i] * v[i] for i in range(m)))
        v = [sum(A[i][j] * v[j] for j in range(m)) for i in range(m)]
    return coeffs


# fixed start of the Newton solve (one branch of the 4-stage 4th-order 2S family)
_START = (1.23, 0.08, 0.93, 0.45,        # beta_1..beta_4
          0.15, -0.88,                   # delta_2, delta_3   (delta_1 = 1, delta_4 = 1)
          0.07, 0.63, -0.60,             # gamma1_2..gamma1_4 (gamma1_1 = 0)
          0.81, 1.39, 1.26)              # gamma2_2..gamma2_4 (gamma2_1 = 1)


def _unpack(x):
    b1, b2, b3, b4, d2, d3, g12, g13, g14, g22, g23, g24 = x
    one = mp.mpf(1)
    return ([0 * one, g12, g13, g14], [one, g22, g23, g24], [b1, b2, b3, b4], [one, d2, d3, one])


def _residual(x):
    coef = _unpack(x)
    A, b, c, u = lsrk2s_butcher(coef)
    return order4_conditions(A, b, c) + [ui - 1 for ui in u[1:]]


def _jacobian(x, h):
    f0 = _residual(x)
    J = mp.matrix(len(f0), len(x))
    for j in range(len(x)):
        xp = list(x); xp[j] += h
        xm = list(x); xm[j] -= h
        fp, fm = _residual(xp), _residual(xm)
        for i in range(len(f0)):
            J[i, j] = (fp[i] - fm[i]) / (2 * h)
    return f0, J


def lsrk2s_rk4(dps: int = 50):
    """The oracle's 4-stage, 4th-order 2S coefficients (gamma1, gamma2, beta, delta) as mpf.

    With delta_4 fixed the conditions still leave a one-parameter curve of solutions (the
    Jacobian has rank 11 of 12), so Newton steps use the minimum-norm (pseudo-inverse)
    correction: from the fixed start this converges to one definite point of the curve."""
    with mp.workdps(dps + 10):
        x = [mp.mpf(v) for v in _START]
        h = mp.mpf(10) ** (-(dps // 2))
        for _ in range(60):
            f, J = _jacobian(x, h)
            if max(abs(v) for v in f) < mp.mpf(10) ** (-dps):
                break
            U, S, V = mp.svd_r(J)
            smax = max(S)
            dx = [mp.mpf(0)] * len(x)
            for k in range(len(S)):
                if S[k] > smax * mp.mpf(10) ** (-(dps // 2)):
                    coef = -sum(U[i, k] * f[i] for i in range(len(f))) / S[k]
                    for j in range(len(x)):
                        dx[j] += coef * V[k, j]
            x = [xi + di for xi, di in zip(x, dx)]
        else:
            raise RuntimeError("2S order conditions: Newton did not converge")
        return _unpack(x)


@functools.lru_cache(maxsize=1)
def lsrk2s_rk4_float():
    """The same coefficients rounded to FP64 (the values the library receives); computed once."""
    g1, g2, b, d = lsrk2s_rk4()
    return tuple(tuple(float(v) for v in arr) for arr in (g1, g2, b, d))


# ---------------------------------------------------------------------------
# The wave system with dissipation, stepped by the 2S recurrence
# ---------------------------------------------------------------------------


def wave_rhs_ko(phi: np.ndarray, K: np.ndarray, s2, dx3, N: int, g: int, n_iter: int, sigma: float, r: int):
    """F_Phi = K + sum_i Q_i[Phi], F_K = sum_i D2_i Phi + sum_i Q_i[K] on global periodic arrays;
    the Laplacian is the decomposed operator of ``oracle.cfd.wave_rhs``."""
    from oracle import cfd as C
    fp, fk = C.wave_rhs(phi, K, s2, dx3, N, g, n_iter)
    if sigma > 0:
        fp = fp + ko_dissipation(phi, r, sigma, dx3)
        fk = fk + ko_dissipation(K, r, sigma, dx3)
    return fp, fk


def wave_lsrk_step(phi, K, dt, coef, s2, dx3, N, g, n_iter=0, sigma=0.0, r=4):
    """One 2S step of the wave system with Kreiss-Oliger dissipation."""
    return lsrk2s_step((phi, K), dt, coef, lambda st: wave_rhs_ko(st[0], st[1], s2, dx3, N, g, n_iter, sigma, r))


# ---------------------------------------------------------------------------
# Shifted wave system (Eq. toyShiftWaveEqnSys, flat background)
# ---------------------------------------------------------------------------


def shifted_wave_rhs(phi, K, beta, s2, b, dx3, N, g, n_iter, sigma, r):
    """F_Phi = beta . grad Phi + K + sum_i Q_i[Phi], F_K = beta . grad K + Laplacian Phi +
    sum_i Q_i[K] on global periodic (z, y, x) arrays; ``beta`` = (beta^x, beta^y, beta^z) global
    arrays; the advective terms are ``oracle.biased.advect_uniform`` with the biased scheme ``b``."""
    from oracle import biased as B
    from oracle import cfd as C
    fp, fk = wave_rhs_ko(phi, K, s2, dx3, N, g, n_iter, sigma, r)
    bb = [C.global_to_blocks(v, N) for v in beta]
    ap = C.blocks_to_global(B.advect_uniform(C.ghost_fill_3d(phi, N, g), bb, b, dx3, N, g, n_iter))
    ak = C.blocks_to_global(B.advect_uniform(C.ghost_fill_3d(K, N, g), bb, b, dx3, N, g, n_iter))
    return fp + ap, fk + ak


def shifted_wave_lsrk_step(phi, K, beta, dt, coef, s2, b, dx3, N, g, n_iter=0, sigma=0.0, r=4):
    """One 2S step of the shifted wave system with dissipation."""
    return lsrk2s_step((phi, K), dt, coef,
                       lambda st: shifted_wave_rhs(st[0], st[1], beta, s2, b, dx3, N, g, n_iter, sigma, r))


def shifted_wave_1d_operator(D1: np.ndarray, D2: np.ndarray, beta: float) -> np.ndarray:
    """L = [[beta D1, I], [D2, beta D1]] of Eq. sd_wave_ops acting on (Phi, K)."""
    n = D1.shape[0]
    return np.block([[beta * D1, np.eye(n)], [D2, beta * D1]])


def exp_integrate(L: np.ndarray, U0: np.ndarray, t: float) -> np.ndarray:
    """U(t) = exp(t L) U(0): formal solution of the semi-discrete linear system."""
    import scipy.linalg as sl
    return sl.expm(t * L) @ U0


# ---------------------------------------------------------------------------
# Advection with upwinded biased operators (Eq. tr2pde with c = -beta)
# ---------------------------------------------------------------------------


def advect_rhs(u, beta, b, dx3, N, g, n_iter, sigma, r):
    """F = beta . grad u (upwinded, ``oracle.biased.advect_uniform``) + sum_i Q_i[u] on a global
    periodic (z, y, x) array; ``beta`` = (beta^x, beta^y, beta^z) global arrays."""
    from oracle import biased as B
    from oracle import cfd as C
    bb = [C.global_to_blocks(v, N) for v in beta]
    F = C.blocks_to_global(B.advect_uniform(C.ghost_fill_3d(u, N, g), bb, b, dx3, N, g, n_iter))
    if sigma > 0:
        F = F + ko_dissipation(u, r, sigma, dx3)
    return F


def advect_lsrk_step(u, beta, dt, coef, b, dx3, N, g, n_iter=0, sigma=0.0, r=4):
    """One 2S step of u_t = beta . grad u + sum_i Q_i[u]."""
    return lsrk2s_step((u,), dt, coef, lambda st: (advect_rhs(st[0], beta, b, dx3, N, g, n_iter, sigma, r),))[0]


def advect_operator_1d(b, beta: float, n: int, dx: float, N: int, g: int, n_iter: int, sigma: float, r: int):
    """Dense n x n matrix of u -> beta D u + Q u on a periodic line of n/N blocks: D the
    decomposed biased operator upwinded for the right-hand-side term beta d_x (right-biased where
    beta > 0, left-biased where beta < 0; oracle.biased.decomposed_1d with n_iter iterations), Q
    the Kreiss-Oliger term (ko_1d).  Columns are the images of the unit vectors."""
    from oracle import biased as B
    side = -1 if beta > 0 else 1
    I = np.eye(n)
    D = B.decomposed_1d(I, b, side, dx, N, g, n_iter)
    Q = np.stack([ko_1d(I[:, j], 0, r, sigma, dx) for j in range(n)], 1) if sigma > 0 else 0.0
    return beta * D + Q


def fully_discrete_2d(Mx: np.ndarray, My: np.ndarray, U0: np.ndarray, dt: float, nsteps: int) -> np.ndarray:
    """nsteps of a 4-stage 4th-order Runge-Kutta method (every member advances a linear autonomous
    system by R(z) = 1 + z + z^2/2 + z^3/6 + z^4/24, including the 2S method above) for
    U_t = My U + U Mx^T, U indexed (y, x): in the eigenbases of Mx and My the operator is
    diagonal with entries lam_y + lam_x, so U(n dt) = Vy [(Vy^-1 U0 Vx^-T) * R(dt(lam_y+lam_x))^n] Vx^T."""
    lx, Vx = np.linalg.eig(Mx)
    ly, Vy = np.linalg.eig(My)
    Uh = np.linalg.solve(Vy, np.linalg.solve(Vx, U0.T).T)
    z = dt * (ly[:, None] + lx[None, :])
    R = 1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24
    return (Vy @ (Uh * R ** nsteps) @ Vx.T).real

