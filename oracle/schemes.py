"""Scheme design, restated from Sec. "Method" of arXiv 2302.14858.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Everything here works on one derivative stencil at a time.  A stencil is the
generalised multi-derivative ansatz of Eq. mdAnsatz:

    dx^{d_r} alpha^{(d_r)} . f~^{(d_r)}_k  =  sum_I dx^{d_I} alpha^{(d_I)} . f^{(d_I)}_k

with coefficient tuples alpha^{(d_K)}_n, n = -L..R (Eq. coeffTupDefn).

* ``taylor_rows``      the linear Taylor-matching constraints (Eq. Tcons and
                       the worked C_S = 7 example that follows it).
* ``solve_exact``      fully order-matched schemes (C_S = C_T + 1), exact
                       rational arithmetic (Padé P, explicit E and L schemes).
* ``eps_series``       power series of the relative modified-wavenumber
                       error eps(eta) = eta~^{d_r}/eta^{d_r} - 1
                       (Eqs. fdpwerrdef, relmodnormwavnum).
* ``tune``             spectral tuning: minimise int_0^pi gamma |e~|^2 d eta
                       (Eqs. sp_error, optfunc, cutoff weight Eq. gammacut)
                       subject to alpha^{(d_r)}_0 = 1 and the Taylor rows.  The
                       problem is a convex equality-constrained quadratic
                       programme, solved exactly through its KKT system at high
                       precision (the paper used IPOPT; the minimiser is the
                       same point).
* ``centered_closure`` the explicit closure C-bar_{p+1} whose eta^{2p} error
                       constant equals the interior's C_0 and whose
                       eta^{2p+1} term vanishes (Sec. "Domain decomposition:
                       dispersion relation preservation", the two conditions
                       after Eq. errelmodwavecentmatch).

Exact rationals use ``fractions.Fraction``; tuned (transcendental) schemes use
``mpmath`` at 50 significant digits.  mpmath is only needed by ``tune`` and
the mp-valued series; it is imported lazily.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from fractions import Fraction
from math import factorial
from typing import Dict, List, Sequence, Tuple

# ---------------------------------------------------------------------------
# Stencil description (Eq. coeffTupDefn, Eq. mdAnsatz)
# ---------------------------------------------------------------------------


@dataclass(frozen=True)
class Ansatz:
    """Shape of a generalised stencil.

    d_r   degree of the sought derivative (left-hand side).
    lhs   (L, R) extents of alpha^{(d_r)}.
    rhs   tuple of (d_I, L_I, R_I) for each known-sample class I, ordered
          d_0 < d_1 < ... (Eq. mdAnsatz); d_r must not appear among them.
    """

    d_r: int
    lhs: Tuple[int, int]
    rhs: Tuple[Tuple[int, int, int], ...]

    def blocks(self):
        """(d, L, R, is_lhs) for every coefficient tuple, lhs first."""
        out = [(self.d_r, self.lhs[0], self.lhs[1], True)]
        for d, L, R in self.rhs:
            out.append((d, L, R, False))
        return out

    def unknowns(self):
        """List of (d, n, is_lhs): one entry per unknown coefficient."""
        u = []
        for d, L, R, is_lhs in self.blocks():
            for n in range(-L, R + 1):
                u.append((d, n, is_lhs))
        return u

    @property
    def C_S(self) -> int:
        """Number of unknowns, C_S of Sec. "Method"."""
        return len(self.unknowns())


@dataclass
class Scheme:
    """Coefficient tuples of one stencil: coeffs[(d, is_lhs)] = {n: alpha_n}."""

    ansatz: Ansatz
    coeffs: Dict[Tuple[int, bool], Dict[int, object]] = field(default_factory=dict)

    def lhs(self) -> Dict[int, object]:
        return self.coeffs[(self.ansatz.d_r, True)]

    def rhs(self, d: int = 0) -> Dict[int, object]:
        return self.coeffs[(d, False)]

    def lhs_list(self) -> List[object]:
        L, R = self.ansatz.lhs
        return [self.lhs()[n] for n in range(-L, R + 1)]

    def rhs_list(self, d: int = 0) -> List[object]:
        for dd, L, R in self.ansatz.rhs:
            if dd == d:
                return [self.rhs(d)[n] for n in range(-L, R + 1)]
        raise KeyError(d)


def _from_vector(ansatz: Ansatz, x: Sequence[object]) -> Scheme:
    s = Scheme(ansatz)
    for (d, n, is_lhs), v in zip(ansatz.unknowns(), x):
        s.coeffs.setdefault((d, is_lhs), {})[n] = v
    return s


# ---------------------------------------------------------------------------
# Taylor constraints (Eq. Tcons substituted into Eq. mdAnsatz)
# ---------------------------------------------------------------------------


def taylor_rows(ansatz: Ansatz, qmax: int, one=Fraction(1)) -> List[List[object]]:
    """Rows of the linear Taylor-matching conditions for q = 0..qmax.

    Substituting f^{(d_K)}_{k+m} = sum_l (m dx)^l / l! f^{(d_K + l)}_k into
    Eq. mdAnsatz, every term carrying f^{(q)}_k has the factor dx^q, so
    matching the coefficient of f^{(q)}_k gives, for each q,

        sum_I sum_m alpha^{(d_I)}_m m^{q-d_I}/(q-d_I)!
          - sum_n alpha^{(d_r)}_n n^{q-d_r}/(q-d_r)!  = 0,

    where a term is present only when q >= its degree (0^0 = 1).  The
    derivative samples f~^{(d_r)} on the left are exact derivatives for this
    truncation-error analysis.
    """
    rows = []
    for q in range(qmax + 1):
        row = []
        for d, n, is_lhs in ansatz.unknowns():
            if q < d:
                row.append(0 * one)
                continue
            c = one * Fraction(n) ** (q - d) / factorial(q - d) if isinstance(one, Fraction) \
                else one * (n ** (q - d)) / factorial(q - d)
            row.append(-c if is_lhs else c)
        rows.append(row)
    return rows


def normalization_row(ansatz: Ansatz, one=Fraction(1)) -> List[object]:
    """The scaling freedom is fixed by alpha^{(d_r)}_0 = 1 (Sec. "Method")."""
    return [one if (is_lhs and n == 0) else 0 * one for d, n, is_lhs in ansatz.unknowns()]


def _exact_solve(rows: List[List[Fraction]], rhs: List[Fraction]) -> List[Fraction]:
    """Gauss-Jordan elimination on an exact, consistent system.

    The system may be over-determined (e.g. odd Taylor rows of a symmetric
    second-derivative stencil are dependent); the solution must be unique.
    """
    m = [list(r) + [b] for r, b in zip(rows, rhs)]
    nrow, ncol = len(m), len(rows[0])
    piv_cols = []
    r = 0
    for c in range(ncol):
        p = next((i for i in range(r, nrow) if m[i][c] != 0), None)
        if p is None:
            continue
        m[r], m[p] = m[p], m[r]
        pv = m[r][c]
        m[r] = [v / pv for v in m[r]]
        for i in range(nrow):
            if i != r and m[i][c] != 0:
                f = m[i][c]
                m[i] = [a - f * b for a, b in zip(m[i], m[r])]
        piv_cols.append(c)
        r += 1
        if r == nrow:
            break
    if len(piv_cols) != ncol:
        raise ValueError("constraints do not determine the stencil uniquely")
    for i in range(r, nrow):
        if m[i][-1] != 0:
            raise ValueError("inconsistent constraints")
    x = [Fraction(0)] * ncol
    for i, c in enumerate(piv_cols):
        x[c] = m[i][-1]
    return x


def solve_exact(ansatz: Ansatz, order: int) -> Scheme:
    """Fully Taylor-matched scheme of formal order ``order`` (C_S = C_T + 1).

    Formal order p means the approximant error is O(dx^p), which needs the
    Taylor rows q = 0 .. p + d_r - 1 (the worked example of Sec. "Method",
    d_r = 1 with rows q = 0..5, is of order dx^5).
    """
    rows = taylor_rows(ansatz, order + ansatz.d_r - 1)
    rhs = [Fraction(0)] * len(rows)
    rows.append(normalization_row(ansatz))
    rhs.append(Fraction(1))
    return _from_vector(ansatz, _exact_solve(rows, rhs))


# ---------------------------------------------------------------------------
# Power series of the modified wavenumber (Eqs. fdpwerrdef, relmodnormwavnum)
# ---------------------------------------------------------------------------


class QQi:
    """Exact complex rational a + b i (enough for series arithmetic)."""

    __slots__ = ("re", "im")

    def __init__(self, re=0, im=0):
        self.re = Fraction(re)
        self.im = Fraction(im)

    def __add__(self, o):
        o = _qqi(o)
        return QQi(self.re + o.re, self.im + o.im)

    __radd__ = __add__

    def __sub__(self, o):
        o = _qqi(o)
        return QQi(self.re - o.re, self.im - o.im)

    def __rsub__(self, o):
        return _qqi(o) - self

    def __mul__(self, o):
        o = _qqi(o)
        return QQi(self.re * o.re - self.im * o.im, self.re * o.im + self.im * o.re)

    __rmul__ = __mul__

    def __truediv__(self, o):
        o = _qqi(o)
        den = o.re * o.re + o.im * o.im
        return QQi((self.re * o.re + self.im * o.im) / den, (self.im * o.re - self.re * o.im) / den)

    def __neg__(self):
        return QQi(-self.re, -self.im)

    def __eq__(self, o):
        o = _qqi(o)
        return self.re == o.re and self.im == o.im

    def __repr__(self):
        return f"QQi({self.re}, {self.im})"


def _qqi(v):
    return v if isinstance(v, QQi) else QQi(v, 0)


def _unit(kind):
    """(one, i) for the requested number field."""
    if kind == "exact":
        return QQi(1), QQi(0, 1)
    import mpmath as mp
    return mp.mpc(1), mp.mpc(0, 1)


def _series_mul(a, b, n):
    return [sum((a[i] * b[k - i] for i in range(k + 1)), a[0] * 0) for k in range(n)]


def _series_div(a, b, n):
    """a / b as power series; b[0] must be non-zero."""
    q = []
    for k in range(n):
        s = a[k]
        for i in range(k):
            s = s - q[i] * b[k - i]
        q.append(s / b[0])
    return q


def _phase_series(coeffs: Dict[int, object], nterms: int, one, i_unit):
    """Series of alpha . E = sum_n alpha_n exp(i n eta) (Eq. phase_tup)."""
    out = [one * 0 for _ in range(nterms)]
    for n, a in coeffs.items():
        term = one * 1
        for k in range(nterms):
            if k > 0:
                term = term * (i_unit * n) / k
            out[k] = out[k] + term * a
    return out


def eps_series(scheme: Scheme, nterms: int = 14, kind: str = "exact"):
    """Series coefficients c_j of eps(eta) = sum_j c_j eta^j.

    (i eta~)^{d_r} = (alpha^{(d_r)} . E)^{-1} sum_I (i eta)^{d_I} alpha^{(d_I)} . E
    (Eq. fdpwerrdef) and eps = eta~^{d_r} / eta^{d_r} - 1 (Eq. relmodnormwavnum).
    Returned values are complex (QQi for kind="exact", mpc for kind="mp").
    """
    if kind != "exact":
        import mpmath as mp
        with mp.workdps(50):
            return _eps_series(scheme, nterms, kind)
    return _eps_series(scheme, nterms, kind)


def _eps_series(scheme: Scheme, nterms: int, kind: str):
    one, i_unit = _unit(kind)
    a = scheme.ansatz
    extra = a.d_r
    n = nterms + extra + 1
    num = [one * 0 for _ in range(n)]
    for d, L, R in a.rhs:
        ser = _phase_series(scheme.rhs(d), n, one, i_unit)
        ipow = one
        for _ in range(d):
            ipow = ipow * i_unit
        for k in range(n - d):
            num[k + d] = num[k + d] + ipow * ser[k]
    den = _phase_series(scheme.lhs(), n, one, i_unit)
    ratio = _series_div(num, den, n)          # (i eta~)^{d_r}
    ipow = one
    for _ in range(a.d_r):
        ipow = ipow * i_unit                  # i^{d_r}
    # eta~^{d_r} / eta^{d_r} = ratio / (i eta)^{d_r}
    lead = ratio[: a.d_r]
    for v in lead:
        if (v.re != 0 or v.im != 0) if kind == "exact" else abs(v) > 1e-25:
            raise ValueError("scheme is not consistent with the derivative degree")
    out = [ratio[k + a.d_r] / ipow for k in range(nterms)]
    out[0] = out[0] - one
    return out


def error_constant(scheme: Scheme, order: int, kind: str = "exact"):
    """Leading constant C_p of eps(eta) ~ C_p eta^p (Eq. adv_ppw_estimate)."""
    ser = eps_series(scheme, order + 2, kind)
    return ser[order]


def modified_wavenumber(scheme: Scheme, eta):
    """eta~(eta) for a real eta, FP64 complex (Eq. fdpwerrdef).

    Returns (i eta~)^{d_r} / i^{d_r} = eta~^{d_r}; callers take the d_r-th root
    where they need eta~ itself.
    """
    import cmath
    a = scheme.ansatz
    num = 0j
    for d, L, R in a.rhs:
        s = sum(complex(float(v)) * cmath.exp(1j * n * eta) for n, v in scheme.rhs(d).items())
        num += (1j * eta) ** d * s
    den = sum(complex(float(v)) * cmath.exp(1j * n * eta) for n, v in scheme.lhs().items())
    return num / den / (1j ** a.d_r)


# ---------------------------------------------------------------------------
# Spectral tuning (Eqs. sp_error, optfunc, gammacut) as a KKT system
# ---------------------------------------------------------------------------


def tune(ansatz: Ansatz, order: int, eta_c, dps: int = 50) -> Scheme:
    """Tuned scheme: argmin int_0^{eta_c} |e~(eta)|^2 d eta under the constraints.

    e~(eta) = sum_I (i eta)^{d_I} E^{(d_I)} . alpha^{(d_I)}
              - (i eta)^{d_r} E^{(d_r)} . alpha^{(d_r)}          (Eq. sp_error)
    The cutoff weight gamma(eta; eta_c) = 1 on [0, eta_c], 0 beyond
    (Eq. gammacut), so the functional of Eq. optfunc is the integral over
    [0, eta_c].  e~ is linear in the unknowns x, e~ = sum_u x_u phi_u(eta), so
    the functional is x^T H x with H_uv = int Re(conj(phi_u) phi_v) d eta.
    Constraints C x = b are alpha^{(d_r)}_0 = 1 and the Taylor rows q = 0 ..
    order + d_r - 1.  The stationarity conditions 2 H x + C^T lam = 0,
    C x = b form one linear system, solved here at ``dps`` digits.  (The
    paper's W-enlargement of Eqs. Wdefn / Zcons, followed by zeroing the extra
    coefficients, describes the same feasible set.)
    """
    import mpmath as mp

    with mp.workdps(dps):
        eta_c = mp.mpf(eta_c)
        unk = ansatz.unknowns()
        nu = len(unk)

        def phi(u, eta):
            d, n, is_lhs = unk[u]
            v = (mp.mpc(0, 1) * eta) ** d * mp.expj(n * eta)
            return -v if is_lhs else v

        H = mp.matrix(nu, nu)
        for u in range(nu):
            for v in range(u, nu):
                val = mp.quad(lambda e: mp.re(mp.conj(phi(u, e)) * phi(v, e)), [0, eta_c])
                H[u, v] = val
                H[v, u] = val
        rows = taylor_rows(ansatz, order + ansatz.d_r - 1, one=mp.mpf(1))
        rows.append(normalization_row(ansatz, one=mp.mpf(1)))
        b = [mp.mpf(0)] * (len(rows) - 1) + [mp.mpf(1)]
        # Drop linearly dependent constraint rows (e.g. odd Taylor rows of a
        # symmetric stencil), keeping an independent set.
        rows, b = _independent_rows(rows, b)
        nc = len(rows)
        K = mp.matrix(nu + nc, nu + nc)
        rhs = mp.matrix(nu + nc, 1)
        for u in range(nu):
            for v in range(nu):
                K[u, v] = 2 * H[u, v]
        for c in range(nc):
            for u in range(nu):
                K[nu + c, u] = rows[c][u]
                K[u, nu + c] = rows[c][u]
            rhs[nu + c] = b[c]
        sol = mp.lu_solve(K, rhs)
        x = [sol[u] for u in range(nu)]
    return _from_vector(ansatz, x)


def _independent_rows(rows, b):
    import mpmath as mp
    kept, kb = [], []
    basis = []
    for r, bb in zip(rows, b):
        v = [mp.mpf(x) for x in r]
        for bv, pc in basis:
            f = v[pc] / bv[pc]
            v = [a - f * c for a, c in zip(v, bv)]
        piv = max(range(len(v)), key=lambda i: abs(v[i]))
        if abs(v[piv]) > mp.mpf(10) ** (-(mp.mp.dps // 2)):
            basis.append((v, piv))
            kept.append(r)
            kb.append(bb)
    return kept, kb


# ---------------------------------------------------------------------------
# Explicit closures with matched error constant (Sec. domdec_drp)
# ---------------------------------------------------------------------------


def centered_closure(interior: Scheme, order: int, halfwidth: int, kind: str = "exact") -> Scheme:
    """Explicit centred closure C-bar_{p+1} for a centred interior scheme.

    ``order`` = 2p is the interior's formal order and ``halfwidth`` = p + 1.
    The closure is an explicit stencil (alpha^{(d_r)} = (1)) with
    alpha^{(0)}_m, m = -halfwidth..halfwidth, fixed by
      * the Taylor rows q = 0 .. 2p + d_r - 1 (formal order 2p);
      * eps coefficient of eta^{2p} equal to the interior's C_0
        (Eq. errrelmodwavcent / errelmodwavecentmatch);
      * eps coefficient of eta^{2p+1} equal to zero.
    For an explicit stencil the eps coefficient of eta^j is
    i^j sum_m alpha_m m^{j+d_r}/(j+d_r)!, so both extra conditions are linear.
    """
    if kind != "exact":
        import mpmath as mp
        with mp.workdps(50):
            return _centered_closure(interior, order, halfwidth, kind)
    return _centered_closure(interior, order, halfwidth, kind)


def _centered_closure(interior: Scheme, order: int, halfwidth: int, kind: str) -> Scheme:
    d_r = interior.ansatz.d_r
    C0 = error_constant(interior, order, kind)
    ans = Ansatz(d_r, (0, 0), ((0, halfwidth, halfwidth),))
    if kind == "exact":
        one = Fraction(1)
        C0r = C0.re
        assert C0.im == 0
    else:
        import mpmath as mp
        one = mp.mpf(1)
        C0r = mp.re(C0)
    rows = taylor_rows(ans, order + d_r - 1, one=one)
    b = [0 * one] * len(rows)
    # condition on eta^{2p}: i^{2p} sum alpha_m m^{2p+d_r}/(2p+d_r)! = C0
    for j, target in ((order, C0r), (order + 1, 0 * one)):
        q = j + d_r
        row = []
        for d, n, is_lhs in ans.unknowns():
            if is_lhs:
                row.append(0 * one)
            else:
                row.append(one * (Fraction(n) ** q if kind == "exact" else n ** q) / factorial(q))
        sign = (-1) ** (j // 2) if j % 2 == 0 else 1
        rows.append(row)
        b.append(target * sign)
    rows.append(normalization_row(ans, one=one))
    b.append(one)
    if kind == "exact":
        x = _exact_solve(rows, b)
    else:
        import mpmath as mp
        rows, b = _independent_rows(rows, b)
        A = mp.matrix(rows)
        x = list(mp.lu_solve(A, mp.matrix(b)))
    return _from_vector(ans, x)


# ---------------------------------------------------------------------------
# Named schemes of the appendix (Tabs. misc_explicit, pade_deg_one/two,
# num_deg_one/two)
# ---------------------------------------------------------------------------


def pade(d_r: int, M: int) -> Scheme:
    """(d_r)P^1_M: tridiagonal left side, 2M+1 function samples, order 2M+2."""
    return solve_exact(Ansatz(d_r, (1, 1), ((0, M, M),)), 2 * M + 2)


def explicit(d_r: int, M: int) -> Scheme:
    """(d_r)E_M: explicit centred, order 2M (Tab. misc_explicit)."""
    return solve_exact(Ansatz(d_r, (0, 0), ((0, M, M),)), 2 * M)


def lopsided(L: int, R: int, order: int) -> Scheme:
    """(1)L_{L,R}: explicit first derivative, L points left, R right."""
    return solve_exact(Ansatz(1, (0, 0), ((0, L, R),)), order)


def tuned_Q(d_r: int, eta_c, lhs=(1, 1), rhs=(3, 3), order: int = 6, dps: int = 50) -> Scheme:
    """(d_r)Q^{lhs}_{rhs}[eta_c]: order-6 scheme tuned with the cutoff eta_c."""
    return tune(Ansatz(d_r, tuple(lhs), ((0, rhs[0], rhs[1]),)), order, eta_c, dps)


def to_float_tuple(values) -> Tuple[float, ...]:
    """Round exact or mp values to the nearest FP64."""
    out = []
    for v in values:
        if isinstance(v, Fraction):
            out.append(v.numerator / v.denominator if abs(v.numerator) < 2 ** 53 and v.denominator < 2 ** 53
                       else float(v))
        else:
            try:
                import mpmath as mp
                if isinstance(v, (mp.mpf, mp.mpc)):
                    out.append(float(mp.re(v)))
                    continue
            except ImportError:
                pass
            out.append(float(v))
    return tuple(out)
