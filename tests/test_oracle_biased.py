"""Pins of oracle/biased.py: the biased UCD / CCU schemes against the printed tables
(Tabs. ucd_slow, ucd_fast, ucd_slow_closure, ucd_fast_closure, ccux_deg_one_col), and
the block systems (Eqs. closure_left_X, iter_left_X) against closed forms, polynomial
exactness, the global scheme and the reflection symmetry."""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import biased as B
from oracle import schemes as SC
from tests.helpers import SCHEMES, rel_max

HERE = os.path.dirname(os.path.abspath(__file__))
PAPER = json.load(open(os.path.join(HERE, "golden", "paper_tables.json")))


def _fr(s):
    return Fraction(s)


def _eps_ok(scheme, printed):
    n = max(int(k) for k in printed) + 2
    e = SC.eps_series(scheme, n)
    for k, (re, im) in printed.items():
        assert e[int(k)] == SC.QQi(_fr(re), _fr(im)), (k, e[int(k)], re, im)


@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_ucd_slow_reproduces_table(M):
    row = PAPER["ucd_slow"]["rows"][str(M)]
    U = B.ucd_slow(M)
    assert U.lhs_list() == [_fr(v) for v in row["lhs"]]
    assert U.rhs_list(0) == [_fr(v) for v in row["rhs"]]
    assert U.rhs_list(2) == [_fr(row["a2"])]
    _eps_ok(U, row["eps"])


@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_ucd_fast_reproduces_table(M):
    row = PAPER["ucd_fast"]["rows"][str(M)]
    V = B.ucd_fast(M)
    assert V.lhs_list() == [_fr(v) for v in row["lhs"]]
    assert V.rhs_list(0) == [_fr(v) for v in row["rhs"]]
    _eps_ok(V, row["eps"])


@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_xi_closures_reproduce_tables(M):
    for key, fn in (("ucd_slow_closure", B.ucd_slow_closure), ("ucd_fast_closure", B.ucd_fast_closure)):
        row = PAPER[key]["rows"][str(M)]
        xi, clo = fn(M)
        assert xi == _fr(row["xi"]), (key, xi)
        _eps_ok(clo, row["eps"])
        # the closure keeps the formal order: Taylor rows through the order hold exactly
        assert clo.lhs() == {0: 1, 1: B.ucd_slow(M).lhs()[-1] if key == "ucd_slow_closure" else B.ucd_fast(M).lhs()[-1]}


def test_xi_closure_plus_side_is_the_negated_xi():
    """xi_+ = -xi_- (Tabs. ucd_slow_closure, ucd_fast_closure): closing the mirrored
    (right-biased) scheme at k*_+ by the same construction, mirrored, gives -xi."""
    for M in (1, 2):
        for interior, n in ((B.ucd_slow(M), 2 * M + 4), (B.ucd_fast(M), 2 * M + 2)):
            xi_m, _ = B.xi_closure(interior, n)
            # right-biased scheme reflected is the left-biased one: build the closure of the
            # reflected problem directly in the right-biased frame
            right = B.mirror(interior)
            base = B.mirror(right)                       # the left-biased scheme at k*_+
            j = n - 1
            target = SC.eps_series(right, j + 2)[j]
            e0 = SC.eps_series(B._with_xi(base, n, Fraction(0)), j + 2)[j]
            e1 = SC.eps_series(B._with_xi(base, n, Fraction(1)), j + 2)[j]
            s = e1 - e0
            xi_p = (target.im - e0.im) / s.im if s.im != 0 else (target.re - e0.re) / s.re
            assert xi_p == -xi_m


@pytest.mark.parametrize("M", [1, 2, 3])
def test_ccu_x_reproduces_table(M):
    row = PAPER["ccux_deg_one_col"]["rows"][str(M)]
    X, xi, Xb = B.ccu_x(M, _fr(row["sigma"]))
    assert X.lhs() == {-1: _fr(row["lhs_sub"]), 0: 1}
    assert X.rhs(0) == {int(k): _fr(v) for k, v in row["rhs"].items()}
    assert Xb.lhs() == {0: 1, 1: _fr(row["closure_sup"])}
    assert Xb.rhs(0) == {int(k): _fr(v) for k, v in row["closure"].items()}
    _eps_ok(X, row["eps"])
    # the closure matches Re eps exactly and Im eps at the lowest order (Tab. ccux caption)
    e, eb = SC.eps_series(X, 2 * M + 5), SC.eps_series(Xb, 2 * M + 5)
    assert e[2 * M + 2] == eb[2 * M + 2] and e[2 * M + 3] == eb[2 * M + 3]


@pytest.mark.parametrize("M,lam_max,printed", [(1, 1, "37/100"), (2, 1, "86/100"), (3, 2, "146/100")])
def test_ccu_weight_selection_rule_gives_the_printed_sigma(M, lam_max, printed):
    """Sec. domdec_drp: start at lam_max (1; 2 for M = 3) and lower lam until Re eta~ <= eta on
    (0, pi] would fail; the last admissible lam (1/100 steps) is the sigma of
    Tab. ccux_deg_one_col, and lam - 1/100 overestimates eta somewhere."""
    assert B.ccu_lambda(M, lam_max) == Fraction(printed)


@pytest.mark.parametrize("maker", ["U2", "V3", "X2"])
def test_mirror_conjugates_eps(maker):
    """eps[S^+] = eps[S^-]^* (captions of Tabs. ucd_slow, ucd_fast, ccux_deg_one_col)."""
    s = {"U2": lambda: B.ucd_slow(2), "V3": lambda: B.ucd_fast(3),
         "X2": lambda: B.ccu_x(2, Fraction(86, 100))[0]}[maker]()
    e, em = SC.eps_series(s, 12), SC.eps_series(B.mirror(s), 12)
    for a, b in zip(e, em):
        assert a.re == b.re and a.im == -b.im


def test_upwind_schemes_have_nonpositive_imaginary_wavenumber():
    """The S_+ schemes of Sec. "Two dimensional advection" (used where the advection speed
    is positive), X_2^- and Q^{1,0}_{3,4}[1], and the fast V_M^- satisfy Im eta~ <= 0 on
    (0, pi] up to a tiny high-order excursion of the tuned scheme (max 6.9e-6 near
    eta = 0.84, from its eta^7 error term); their mirrors are anti-dissipative there.
    (The slow U_M^- with an exact f^{(2)} is indefinite near eta = pi.)"""
    q, _ = B.tuned_Q1034(1)
    cases = [(B.ccu_x(1, Fraction(37, 100))[0], 1e-14), (B.ccu_x(2, Fraction(86, 100))[0], 1e-14),
             (q, 1e-5)] + [(B.ucd_fast(M), 1e-13) for M in (1, 2, 3)]
    etas = np.linspace(1e-3, np.pi, 400)
    for s, tol in cases:
        im = np.array([SC.modified_wavenumber(s, e).imag for e in etas])
        assert im.max() <= tol
        assert im.min() < -0.5
        imm = np.array([SC.modified_wavenumber(B.mirror(s), e).imag for e in etas])
        assert np.allclose(imm, -im, atol=1e-13)


# ---------------------------------------------------------------------------
# Block systems
# ---------------------------------------------------------------------------


def _biased(name):
    e = SCHEMES[name]
    return B.Biased(e["a"], e["lo"], tuple(e["rhs"]), e["c_sup"], e["c_lo"], tuple(e["closure"]), e["kc"])


@pytest.mark.parametrize("name", ["X1_d1", "X2_d1", "Q1034_1_d1"])
@pytest.mark.parametrize("side", [1, -1])
def test_block_system_is_exact_on_polynomials(name, side):
    """A single block with ghosts sampled from a polynomial of the scheme's formal
    degree: the closed system (closure row + interior rows) returns f' exactly."""
    b = _biased(name)
    order = SCHEMES[name]["order"]
    N, g = 16, 4
    dx = 0.37
    x = (np.arange(-g, N + g) + 0.5) * dx - 2.0
    rng = np.random.default_rng(7)
    c = rng.standard_normal(order + 1)
    f = np.polyval(c, x)
    want = np.polyval(np.polyder(c), x[g:g + N])
    d = B.closed_solve(f[:, None], b, side, dx, N, g)[:, 0]
    assert rel_max(d, want) < 1e-12
    # one degree more is not exact (the closure or the interior has an error term)
    c2 = np.concatenate([[1.0], np.zeros(order + 1)])
    f2 = np.polyval(c2, x)
    d2 = B.closed_solve(f2[:, None], b, side, dx, N, g)[:, 0]
    assert rel_max(d2, np.polyval(np.polyder(c2), x[g:g + N])) > 1e-9


@pytest.mark.parametrize("name", ["X2_d1", "Q1034_1_d1"])
def test_global_scheme_closed_form(name):
    """Circulant global scheme on exp(ikx): multiplication by i eta~(k dx)/dx with eta~
    from Eq. fdpwerrdef evaluated on the exact-rational scheme."""
    b = _biased(name)
    n = 64
    dx = 2 * np.pi / n
    x = (np.arange(n) + 0.5) * dx
    s = {"X2_d1": lambda: B.ccu_x(2, Fraction(86, 100))[0], "Q1034_1_d1": lambda: B.tuned_Q1034(1)[0]}[name]()
    for k in (1, 7, 20):
        f = np.exp(1j * k * x)
        for side, sch in ((1, s), (-1, B.mirror(s))):
            got = B.global_periodic(f.real, b, side, dx) + 1j * B.global_periodic(f.imag, b, side, dx)
            want = 1j * SC.modified_wavenumber(sch, k * dx) / dx * f
            assert np.max(np.abs(got - want)) < 1e-11 * np.max(np.abs(want))


@pytest.mark.parametrize("name", ["X2_d1", "Q1034_1_d1"])
@pytest.mark.parametrize("side", [1, -1])
def test_iteration_converges_to_the_global_scheme(name, side):
    """Fixed point of Eq. iter_left_X is the undecomposed scheme; the biased iteration
    saturates fast (Sec. domdec_iter: one iteration reaches saturation)."""
    b = _biased(name)
    NM, N, g = 64, 16, 4
    dx = 2 * np.pi / NM
    x = (np.arange(NM) + 0.5) * dx
    f = 0.05 * np.exp(-np.sin(2 * (x - 0.2)))          # g of Eq. test_grid_conv_g
    ref = B.global_periodic(f, b, side, dx)
    errs = [rel_max(B.decomposed_1d(f, b, side, dx, N, g, i), ref) for i in range(4)]
    assert errs[0] > 1e-8
    assert errs[1] < errs[0] * 1e-2
    assert errs[3] < 1e-13


@pytest.mark.parametrize("n_iter", [0, 1])
def test_right_biased_is_the_reflection_of_left_biased(n_iter):
    """D[S_-] f (x) = -D[S_+] (f reflected) (reflected x): checks the mirrored closure
    row at k*_+ and the right-sided iteration node against the left-biased system."""
    b = _biased("X2_d1")
    NM, N, g = 64, 16, 4
    dx = 2 * np.pi / NM
    rng = np.random.default_rng(3)
    f = rng.standard_normal(NM)
    dm = B.decomposed_1d(f, b, -1, dx, N, g, n_iter)
    dp_ref = B.decomposed_1d(f[::-1].copy(), b, +1, dx, N, g, n_iter)
    assert rel_max(dm, -dp_ref[::-1]) < 1e-13


def test_upwind_choice_is_stable_and_the_opposite_is_not():
    """Semi-discrete advection u_t = -c D u (Sec. "Two dimensional advection"): with the
    upwind choice S_+ for c > 0 every eigenvalue has Re <= 0; S_- for c > 0 does not."""
    b = _biased("X2_d1")
    n = 32
    dx = 2 * np.pi / n
    for side, stable in ((1, True), (-1, False)):
        A, Bm = B.cyclic_matrices(b, side, n, dx)
        lam = np.linalg.eigvals(-np.linalg.solve(A, Bm))
        if stable:
            assert lam.real.max() < 1e-12
        else:
            assert lam.real.max() > 1e-3


def test_shift_term_upwinding_is_stable_and_the_opposite_is_not():
    """The right-hand-side term beta d_x u with the upwinding of advect_uniform (right-biased
    where beta > 0, left-biased where beta < 0) has no growing mode for either sign of beta;
    the opposite choice has eigenvalues with Re > 0."""
    b = _biased("X2_d1")
    n = 32
    dx = 2 * np.pi / n
    for beta in (0.7, -0.7):
        good = -1 if beta > 0 else 1
        for side, stable in ((good, True), (-good, False)):
            A, Bm = B.cyclic_matrices(b, side, n, dx)
            lam = np.linalg.eigvals(beta * np.linalg.solve(A, Bm))
            if stable:
                assert lam.real.max() < 1e-12
            else:
                assert lam.real.max() > 1e-3


def test_advect_uniform_selects_the_upwind_side_pointwise():
    """Eq. biasderapproxadv with a pointwise shift of both signs (c = -beta): where beta^x > 0
    the term equals beta^x times the right-biased derivative, where beta^x < 0 the left-biased
    one; beta^y = beta^z = 0.  Converged iteration = the global schemes."""
    b = _biased("Q1034_1_d1")
    NM, N, g = 32, 16, 4
    dx = 2 * np.pi / NM
    x = (np.arange(NM) + 0.5) * dx
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    f = np.sin(6 * X + 0.3) * np.cos(2 * Y) + 0.2 * np.sin(3 * Z)
    from oracle import cfd as C
    ext = C.ghost_fill_3d(f, N, g)
    bx = np.cos(X + 2 * Z)                               # both signs
    zero = np.zeros_like(bx)
    beta = [C.global_to_blocks(v, N) for v in (bx, zero, zero)]
    got = C.blocks_to_global(B.advect_uniform(ext, beta, b, (dx, dx, dx), N, g, n_iter=4))
    dp = np.moveaxis(B.global_periodic(np.moveaxis(f, 2, 0), b, +1, dx), 0, 2)
    dm = np.moveaxis(B.global_periodic(np.moveaxis(f, 2, 0), b, -1, dx), 0, 2)
    want = np.where(bx > 0, bx * dm, bx * dp)
    assert rel_max(got, want) < 1e-12
    # the swapped choice is measurably different
    assert rel_max(np.where(bx > 0, bx * dp, bx * dm), want) > 1e-6
