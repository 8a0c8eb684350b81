"""Biased (upwind) first-degree compact schemes and their block systems.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Restated from Sec. "Domain decomposition: dispersion relation preservation",
Sec. "Domain decomposition: iteration of closures" and Sec. "Two dimensional
advection" of arXiv 2302.14858.

Scheme design (exact rationals, ``oracle.schemes`` machinery)
--------------------------------------------------------------
* ``ucd_slow(M)``  U_M^-: Eq. defChenSchemes with left-biased left side
  (alpha^{(1)}_{-1}, alpha^{(1)}_0), function samples m = -M..M and the
  second-derivative term dx alpha^{(2)}_0 f^{(2)}_k, Taylor-matched to order
  2M+2 (Tab. ucd_slow).
* ``ucd_fast(M)``  V_M^-: the same without the f^{(2)} term, order 2M+1
  (Tab. ucd_fast).
* ``mirror``       the oppositely biased scheme: alpha^{(1)}_m -> alpha^{(1)}_{-m},
  alpha^{(d_I)}_m -> (-1)^{d_I + 1} alpha^{(d_I)}_{-m} (first-degree schemes;
  the rule stated with Tabs. ucd_slow, ucd_fast, ccux_deg_one_col).
* ``xi_closure``   the single-point closure at k*_- of a left-biased scheme:
  the mirrored scheme plus xi dx^n alpha^{(1)}[mirror] . f^{(n)}, with f^{(n)}
  approximated by the centred explicit (n)E_{n/2} (Tab. diss_scheme), and xi
  fixed so that the closure's eps coefficient at eta^{n-1} equals the
  interior's (Eqs. ucd_slow_closure_chi, ucd_fast_closure_chi and the
  matching conditions after them).  Reading: for U_M the term that moves the
  eta^{2M+3} coefficient is n = 2M+4; n = 2M+2 as printed in
  Eq. ucd_slow_closure_chi would change the order of the scheme (and the
  printed xi of Tab. ucd_slow_closure are reproduced only with n = 2M+4).
  For V_M, n = 2M+2 as printed.
* ``ccu_x(M, lam)`` the CCU(M, M+1) scheme X_M^- of Eq. LCslowfast with the
  embedded f^{(2)} approximated by (2)E_{M+2}:  lam U_M^- + (1 - lam) V_{M+1}^-,
  and its closure X-bar_M^- = the xi closure of X_M^- with n = 2M+4
  (Tab. ccux_deg_one_col; lam is the tabulated sigma).
* ``ccu_lambda(M, lam_max)`` the weight selection rule of Sec. domdec_drp (lam_max = 1, or 2
  for M = 3 where the combination overestimates eta at lam <= 1); reading: lam is lowered in
  steps of 1/100 (the printed precision) while Re eta~ <= eta holds on (0, pi].

Block systems (FP64, numpy)
---------------------------
A left-biased scheme on a block of N interior points (local k = 0..N-1,
k*_- = 0, k*_+ = N-1, ghosts g) is solved as Eq. closure_left_X: row k*_- is
the closure (alpha-bar_0 = 1 at k, alpha-bar_{+1} at k+1), rows k = 1..N-1 the
interior scheme (alpha_{-1} at k-1, 1 at k).  Its mirror (the right-biased
scheme) uses the interior rows k = 0..N-2 and the mirrored closure at k*_+.
The hybrid iteration is Eq. iter_left_X: with k^c_- = k*_- - kc the unknown
at k^c_- is the neighbour's previous iterate and rows k^c_- + 1 .. k*_+ are
the interior scheme (right-biased: k^c_+ = k*_+ + kc, rows k*_- .. k^c_+ - 1).
Each system is assembled as a dense N x N (or (N+kc) x (N+kc)) matrix and
solved with the library dense solver.

Upwinding (Eq. biasderapproxadv, Sec. "Two dimensional advection" and Sec.
"Z4c: system description"): in u_t + c u_x = 0 the term c D u takes S_+ (the
scheme with Im eta~ <= 0, here the left-biased one) where c > 0 and S_- (its
mirror) where c < 0, so that the semi-discrete operator -c D has no growing
modes.  Reading: as printed the weights (|c| -+ c)/2 multiply D without the sign
of c, which does not reduce to c D for c < 0; the reading is the split
c_+ D[S_+] + c_- D[S_-], c_+- = (c +- |c|)/2.  A shift-advection term
beta^i d_i u on the right-hand side (u_t = beta^i d_i u + ...) transports with
velocity c = -beta^i, so it becomes
    beta^i_- D_i[S_+] u + beta^i_+ D_i[S_-] u,   beta_+- = (beta +- |beta|)/2:
the right-biased scheme where beta^i > 0 and the left-biased one where
beta^i < 0.  (Taking c = +beta^i instead makes the operator anti-dissipative:
the pin below shows eigenvalues with Re > 0, and an evolution grows without
bound.)
"""
from __future__ import annotations

from dataclasses import dataclass
from fractions import Fraction
from typing import Dict, Sequence, Tuple

import numpy as np

from oracle import schemes as SC

# ---------------------------------------------------------------------------
# Scheme design
# ---------------------------------------------------------------------------


def ucd_slow(M: int) -> SC.Scheme:
    """U_M^- of Tab. ucd_slow (Eq. defChenSchemes with the f^{(2)} term)."""
    return SC.solve_exact(SC.Ansatz(1, (1, 0), ((0, M, M), (2, 0, 0))), 2 * M + 2)


def ucd_fast(M: int) -> SC.Scheme:
    """V_M^- of Tab. ucd_fast (Eq. defChenSchemes without the f^{(2)} term)."""
    return SC.solve_exact(SC.Ansatz(1, (1, 0), ((0, M, M),)), 2 * M + 1)


def _make(d_r: int, lhs: Dict[int, object], rhs: Dict[int, Dict[int, object]]) -> SC.Scheme:
    """Scheme from coefficient dictionaries (degree -> {offset: value}); offsets
    missing inside a stencil's extent are zero."""
    L, R = -min(lhs), max(lhs)
    zero = 0 * next(iter(lhs.values()))
    classes = tuple((d, -min(c), max(c)) for d, c in sorted(rhs.items()))
    s = SC.Scheme(SC.Ansatz(d_r, (L, R), classes))
    s.coeffs[(d_r, True)] = {n: lhs.get(n, zero) for n in range(-L, R + 1)}
    for d, cl, cr in classes:
        s.coeffs[(d, False)] = {m: rhs[d].get(m, zero) for m in range(-cl, cr + 1)}
    return s


def _rhs_dicts(s: SC.Scheme) -> Dict[int, Dict[int, object]]:
    return {d: dict(s.rhs(d)) for d, _, _ in s.ansatz.rhs}


def mirror(s: SC.Scheme) -> SC.Scheme:
    """Oppositely biased first-degree scheme: reflect x -> -x and multiply the
    relation by -1, so alpha^{(1)}_m -> alpha^{(1)}_{-m} and a right-hand class
    of degree d_I picks up (-1)^{d_I + 1}."""
    assert s.ansatz.d_r == 1
    lhs = {-n: v for n, v in s.lhs().items()}
    rhs = {d: {-m: (-1) ** (d + 1) * v for m, v in c.items()} for d, c in _rhs_dicts(s).items()}
    return _make(1, lhs, rhs)


def explicit_even(n: int) -> SC.Scheme:
    """(n)E_{n/2}: centred explicit approximant of f^{(n)} on n + 1 points,
    order dx^2 (Tab. diss_scheme)."""
    h = n // 2
    return SC.solve_exact(SC.Ansatz(n, (0, 0), ((0, h, h),)), 2)


def embed_second(s: SC.Scheme, M2: int) -> SC.Scheme:
    """Replace dx alpha^{(2)}_0 f^{(2)}_k by dx^{-1} alpha^{(2)}_0 sum_m e_m f_{k+m},
    e = (2)E_{M2} (Sec. domdec_drp, the X_M construction)."""
    e = SC.explicit(2, M2).rhs(0)
    rhs = _rhs_dicts(s)
    a2 = rhs.pop(2)[0]
    r0 = dict(rhs[0])
    for m, v in e.items():
        r0[m] = r0.get(m, 0 * v) + a2 * v
    return _make(1, dict(s.lhs()), {0: r0})


def combine(lam, s1: SC.Scheme, s2: SC.Scheme) -> SC.Scheme:
    """lam s1 + (1 - lam) s2 on the union of the stencils (Eq. LCslowfast)."""
    out_l: Dict[int, object] = {}
    for w, s in ((lam, s1), (1 - lam, s2)):
        for n, v in s.lhs().items():
            out_l[n] = out_l.get(n, 0 * v) + w * v
    out_r: Dict[int, Dict[int, object]] = {}
    for w, s in ((lam, s1), (1 - lam, s2)):
        for d, c in _rhs_dicts(s).items():
            dst = out_r.setdefault(d, {})
            for m, v in c.items():
                dst[m] = dst.get(m, 0 * v) + w * v
    return _make(1, out_l, out_r)


def _with_xi(base: SC.Scheme, n: int, xi) -> SC.Scheme:
    """base + xi dx^n alpha^{(1)}[base] . f^{(n)} with f^{(n)} ~ (n)E_{n/2}: the
    term sum_j alpha_j f^{(n)}_{k+j} adds xi alpha_j e_m to the function
    coefficient at offset j + m."""
    e = explicit_even(n).rhs(0)
    rhs = _rhs_dicts(base)
    r0 = dict(rhs[0])
    for j, a in base.lhs().items():
        for m, v in e.items():
            r0[j + m] = r0.get(j + m, 0 * v) + xi * a * v
    rhs[0] = r0
    return _make(1, dict(base.lhs()), rhs)


def xi_closure(interior: SC.Scheme, n: int) -> Tuple[object, SC.Scheme]:
    """(xi, closure at k*_-) for a left-biased interior scheme (Eqs.
    ucd_slow_closure_chi / ucd_fast_closure_chi and their matching conditions):
    the eps coefficient at eta^{n-1} of the closure equals the interior's.
    eps is affine in xi, so two evaluations fix it exactly."""
    base = mirror(interior)
    j = n - 1
    target = SC.eps_series(interior, j + 2)[j]
    e0 = SC.eps_series(_with_xi(base, n, Fraction(0)), j + 2)[j]
    e1 = SC.eps_series(_with_xi(base, n, Fraction(1)), j + 2)[j]
    slope = e1 - e0
    # the coefficient is purely imaginary (odd power) or real (even power)
    if slope.im != 0:
        xi = (target.im - e0.im) / slope.im
    else:
        xi = (target.re - e0.re) / slope.re
    clo = _with_xi(base, n, xi)
    chk = SC.eps_series(clo, j + 2)[j]
    assert chk == target
    return xi, clo


def ucd_slow_closure(M: int):
    """U-bar_M^-: xi closure of U_M^- with n = 2M + 4 (reading; Tab. ucd_slow_closure)."""
    return xi_closure(ucd_slow(M), 2 * M + 4)


def ucd_fast_closure(M: int):
    """V-bar_M^-: xi closure of V_M^- with n = 2M + 2 (Tab. ucd_fast_closure)."""
    return xi_closure(ucd_fast(M), 2 * M + 2)


def ccu_x(M: int, lam) -> Tuple[SC.Scheme, object, SC.Scheme]:
    """(X_M^-, xi, X-bar_M^-) of Tab. ccux_deg_one_col for the weight lam."""
    U = embed_second(ucd_slow(M), M + 2)
    X = combine(lam, U, ucd_fast(M + 1))
    xi, Xb = xi_closure(X, 2 * M + 4)
    return X, xi, Xb


def ccu_x_interior(M: int, lam) -> SC.Scheme:
    """X_M^- without its closure: lam U_M^- (f'' from (2)E_{M+2}) + (1 - lam) V_{M+1}^-."""
    return combine(lam, embed_second(ucd_slow(M), M + 2), ucd_fast(M + 1))


def ccu_lambda(M: int, lam_max, step=Fraction(1, 100), n_eta: int = 2000):
    """The weight of Eq. LCslowfast by the selection rule of Sec. domdec_drp: start at lam_max and
    reduce lam (in steps of ``step``) while Re eta~ <= eta holds on (0, pi]; return the last lam
    for which it holds (None if lam_max already fails).  The comparison is on ``n_eta`` points
    with a 1e-12 tolerance."""
    import numpy as np
    etas = np.linspace(1e-3, np.pi, n_eta)

    def ok(lam):
        X = ccu_x_interior(M, lam)
        return max(SC.modified_wavenumber(X, e).real - e for e in etas) <= 1e-12

    lam = Fraction(lam_max)
    if not ok(lam):
        return None
    while lam - step >= 0 and ok(lam - step):
        lam -= step
    return lam


def tuned_Q1034(eta_c=1) -> Tuple[SC.Scheme, SC.Scheme]:
    """((1)Q^{1,0}_{3,4}[eta_c], its closure at k*_-).  The paper tabulates no
    closure for the biased tuned scheme; following the single-point closure of
    Sec. domdec_drp, the oppositely biased scheme (1)Q^{0,1}_{4,3} is imposed
    at k*_- (it has the same Re eta~, so dispersion is preserved)."""
    q = SC.tuned_Q(1, eta_c, lhs=(1, 0), rhs=(3, 4))
    return q, mirror(q)


# ---------------------------------------------------------------------------
# FP64 description consumed by the block solvers
# ---------------------------------------------------------------------------


@dataclass(frozen=True)
class Biased:
    """Left-biased first-degree scheme (interior and closure at k*_-).

    a        alpha^{(1)}_{-1} (alpha^{(1)}_0 = 1)
    lo       first offset of the interior right-hand side; rhs = alpha^{(0)}_{lo..}
    c_sup    closure alpha-bar^{(1)}_{+1} (alpha-bar^{(1)}_0 = 1)
    c_lo     first offset of the closure right-hand side
    kc       iteration node k^c_- = k*_- - kc (Eq. iter_left_X)
    """

    a: float
    lo: int
    rhs: Tuple[float, ...]
    c_sup: float
    c_lo: int
    closure: Tuple[float, ...]
    kc: int

    @property
    def hi(self) -> int:
        return self.lo + len(self.rhs) - 1

    @property
    def c_hi(self) -> int:
        return self.c_lo + len(self.closure) - 1


def to_biased(interior: SC.Scheme, closure: SC.Scheme, kc: int) -> Biased:
    """Round a left-biased interior scheme and its closure to FP64."""
    assert set(interior.lhs()) == {-1, 0} and interior.lhs()[0] == 1
    assert set(closure.lhs()) == {0, 1} and closure.lhs()[0] == 1
    assert [d for d, _, _ in interior.ansatz.rhs] == [0] and [d for d, _, _ in closure.ansatz.rhs] == [0]
    L, _ = interior.ansatz.rhs[0][1:]
    cL, _ = closure.ansatz.rhs[0][1:]
    f = SC.to_float_tuple
    return Biased(a=f([interior.lhs()[-1]])[0], lo=-L, rhs=f(interior.rhs_list()),
                  c_sup=f([closure.lhs()[1]])[0], c_lo=-cL, closure=f(closure.rhs_list()), kc=kc)


# ---------------------------------------------------------------------------
# Block systems
# ---------------------------------------------------------------------------


def _side_coeffs(b: Biased, side: int):
    """(interior lhs {offset: a}, interior rhs {offset: c}, closure lhs, closure rhs)
    for side +1 (the left-biased scheme as given) or -1 (its mirror, by the
    coefficient rule of Tab. ucd_slow)."""
    rhs = {b.lo + i: c for i, c in enumerate(b.rhs)}
    clo = {b.c_lo + i: c for i, c in enumerate(b.closure)}
    if side > 0:
        return {-1: b.a}, rhs, {1: b.c_sup}, clo
    return ({1: b.a}, {-m: -c for m, c in rhs.items()},
            {-1: b.c_sup}, {-m: -c for m, c in clo.items()})


def _stencil(f: np.ndarray, coeffs: Dict[int, float], k: int, g: int) -> np.ndarray:
    """sum_m c_m f_{k+m}, offsets in increasing order (f has index k + g on axis 0)."""
    acc = None
    for m in sorted(coeffs):
        term = coeffs[m] * f[k + m + g]
        acc = term if acc is None else acc + term
    return acc


def closed_solve(f: np.ndarray, b: Biased, side: int, dx: float, N: int, g: int) -> np.ndarray:
    """Eq. closure_left_X (side +1) or its right-biased counterpart (side -1)
    on one block: ``f`` is (N + 2g, ...), returns (N, ...)."""
    il, ir, cl, cr = _side_coeffs(b, side)
    kcl = 0 if side > 0 else N - 1                      # closure row k*_-+
    A = np.eye(N)
    R = np.empty((N,) + f.shape[1:])
    for k in range(N):
        lhs, rhs = (cl, cr) if k == kcl else (il, ir)
        assert min(rhs) + k >= -g and max(rhs) + k <= N - 1 + g
        for j, v in lhs.items():
            A[k, k + j] = v
        R[k] = _stencil(f, rhs, k, g) / dx
    return np.linalg.solve(A, R.reshape(N, -1)).reshape(R.shape)


def iterated_solve(f: np.ndarray, b: Biased, side: int, dx: float, N: int, g: int,
                   d_c: np.ndarray) -> np.ndarray:
    """Eq. iter_left_X (side +1): unknowns k = -kc .. N-1, row -kc fixed to the
    neighbour's previous iterate ``d_c``, rows -kc+1 .. N-1 the interior scheme.
    Side -1: unknowns 0 .. N-1+kc, row N-1+kc fixed, rows 0 .. N-2+kc interior.
    Returns the N interior values."""
    il, ir, _, _ = _side_coeffs(b, side)
    n = N + b.kc
    k0 = -b.kc if side > 0 else 0                      # local index of unknown 0
    fixed = 0 if side > 0 else n - 1
    A = np.eye(n)
    R = np.empty((n,) + f.shape[1:])
    for r in range(n):
        k = k0 + r
        if r == fixed:
            R[r] = d_c
            continue
        assert min(ir) + k >= -g and max(ir) + k <= N - 1 + g
        for j, v in il.items():
            A[r, r + j] = v
        R[r] = _stencil(f, ir, k, g) / dx
    x = np.linalg.solve(A, R.reshape(n, -1)).reshape(R.shape)
    return x[b.kc:] if side > 0 else x[:N]


def cyclic_matrices(b: Biased, side: int, n: int, dx: float):
    """Global periodic (undecomposed) interior scheme as circulant (A, B)."""
    il, ir, _, _ = _side_coeffs(b, side)
    A = np.eye(n)
    B = np.zeros((n, n))
    for k in range(n):
        for j, v in il.items():
            A[k, (k + j) % n] += v
        for m, c in ir.items():
            B[k, (k + m) % n] += c / dx
    return A, B


def global_periodic(fg: np.ndarray, b: Biased, side: int, dx: float) -> np.ndarray:
    n = fg.shape[0]
    A, B = cyclic_matrices(b, side, n, dx)
    return np.linalg.solve(A, B @ fg.reshape(n, -1)).reshape(fg.shape)


def _ghost_fill_1d(fg: np.ndarray, N: int, g: int) -> np.ndarray:
    NM = fg.shape[0]
    NS = NM // N
    idx = (np.arange(NS)[:, None] * N + np.arange(-g, N + g)[None, :]) % NM
    return fg[idx]


def decomposed_1d(fg: np.ndarray, b: Biased, side: int, dx: float, N: int, g: int,
                  n_iter: int) -> np.ndarray:
    """Periodic line under decomposition: [0] closed solves, then n_iter Jacobi
    iterations of Eq. iter_left_X (the k^c node reads the neighbour's [i-1]
    value at the same global point)."""
    ext = _ghost_fill_1d(fg, N, g)
    NS = ext.shape[0]
    d = np.stack([closed_solve(ext[I], b, side, dx, N, g) for I in range(NS)])
    for _ in range(n_iter):
        prev = d
        if side > 0:     # k^c_- = -kc is the left neighbour's local N - kc
            d = np.stack([iterated_solve(ext[I], b, side, dx, N, g, prev[(I - 1) % NS][N - b.kc])
                          for I in range(NS)])
        else:            # k^c_+ = N-1+kc is the right neighbour's local kc - 1
            d = np.stack([iterated_solve(ext[I], b, side, dx, N, g, prev[(I + 1) % NS][b.kc - 1])
                          for I in range(NS)])
    return d.reshape((NS * N,) + fg.shape[1:])


# ---------------------------------------------------------------------------
# 3D: biased derivatives and the upwinded advective term
# ---------------------------------------------------------------------------


def axis_solve(data: np.ndarray, axis: int, b: Biased, side: int, dx: float, N: int, g: int,
               n_iter: int) -> np.ndarray:
    """Biased derivative along local ``axis`` (0 z, 1 y, 2 x) of a uniform
    periodic decomposition ``data`` (nbz, nby, nbx, e0, e1, e2), extent N + 2g
    along ``axis``.  Iteration values come from the periodic neighbour block
    along the same axis."""
    ax = 3 + axis
    f = np.moveaxis(data, ax, 0)
    d = closed_solve(f, b, side, dx, N, g)
    for _ in range(n_iter):
        prev = d
        if side > 0:
            dc = np.roll(prev, 1, axis=1 + axis)[N - b.kc]
        else:
            dc = np.roll(prev, -1, axis=1 + axis)[b.kc - 1]
        d = iterated_solve(f, b, side, dx, N, g, dc)
    return np.moveaxis(d, 0, ax)


def biased_uniform(ext: np.ndarray, b: Biased, side: int, dx3: Sequence[float], N: int, g: int,
                   axes: Sequence[str] = ("x", "y", "z"), n_iter: int = 0) -> Dict[str, np.ndarray]:
    """Biased first derivatives on a uniform periodic decomposition; ``ext`` is
    (nbz, nby, nbx, E, E, E) with ghosts filled; ``dx3`` = (dx_x, dx_y, dx_z)."""
    ax = {"z": 0, "y": 1, "x": 2}
    dxs = {"x": dx3[0], "y": dx3[1], "z": dx3[2]}
    I = slice(g, g + N)
    out = {}
    for c in axes:
        sl = [slice(None)] * 3 + [I, I, I]
        sl[3 + ax[c]] = slice(None)
        out[c] = axis_solve(ext[tuple(sl)], ax[c], b, side, dxs[c], N, g, n_iter)
    return out


def advect_uniform(ext: np.ndarray, beta: Sequence[np.ndarray], b: Biased, dx3: Sequence[float],
                   N: int, g: int, n_iter: int = 0) -> np.ndarray:
    """Upwinded right-hand-side term beta^i d_i f (Eq. biasderapproxadv with c = -beta^i pointwise):
    sum over i = x, y, z (in that order) of beta^i_- D_i[S_+] f + beta^i_+ D_i[S_-] f.
    ``beta`` = (beta^x, beta^y, beta^z), each (nbz, nby, nbx, N, N, N) interior."""
    dp = biased_uniform(ext, b, +1, dx3, N, g, ("x", "y", "z"), n_iter)
    dm = biased_uniform(ext, b, -1, dx3, N, g, ("x", "y", "z"), n_iter)
    out = None
    for c, bc in zip(("x", "y", "z"), beta):
        bp = 0.5 * (bc + np.abs(bc))
        bm = 0.5 * (bc - np.abs(bc))
        term = bm * dp[c] + bp * dm[c]
        out = term if out is None else out + term
    return out
