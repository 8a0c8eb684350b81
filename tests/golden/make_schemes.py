"""Write tests/golden/schemes.json: FP64 coefficients derived by the oracle.

Run from the repository root:  python tests/golden/make_schemes.py

Calls only ``oracle.schemes``.  Padé schemes and their closures are exact
rationals rounded once to FP64; the tuned Q^1_3[eta_c] schemes are the KKT
minimisers of Eq. optfunc (cutoff Eq. gammacut) and the Q-bar_4 closures the
C_0-matched explicit stencils, both computed at 50 digits and rounded once.
The printed appendix values are 8-digit roundings of the same numbers; these
full-precision values satisfy the order conditions to FP64 rounding, which the
printed ones do not (their first-moment residual is ~1e-8).
"""
from __future__ import annotations

import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import biased as BI  # noqa: E402
from oracle import schemes as S  # noqa: E402


def _entry(interior, closure, d, order, kind, cite, eta_c=None):
    C0 = S.error_constant(interior, order, kind)
    return {
        "d": d,
        "order": order,
        "eta_c": eta_c,
        "a": S.to_float_tuple([interior.lhs()[1]])[0],
        "rhs": list(S.to_float_tuple(interior.rhs_list())),
        "closure": list(S.to_float_tuple(closure.rhs_list())),
        "C0": float(C0.re) if kind == "exact" else float(C0.real),
        "cite": cite,
    }


def build() -> dict:
    import mpmath as mp
    out = {"_about": "FP64 scheme coefficients written by tests/golden/make_schemes.py from oracle.schemes"}
    for d, tab in ((1, "Tab. pade_deg_one"), (2, "Tab. pade_deg_two")):
        for M in (1, 2, 3):
            order = 2 * M + 2
            p = S.pade(d, M)
            c = S.centered_closure(p, order, M + 2)
            out[f"P{M}_d{d}"] = _entry(p, c, d, order, "exact", tab)
    for d, tab in ((1, "Tab. num_deg_one"), (2, "Tab. num_deg_two")):
        for name, eta_c in (("1", mp.mpf(1)), ("4pi5", 4 * mp.pi / 5)):
            q = S.tuned_Q(d, eta_c)
            c = S.centered_closure(q, 6, 4, "mp")
            out[f"Q13_{name}_d{d}"] = _entry(q, c, d, 6, "mp", tab, float(eta_c))
    # left-biased first-degree schemes with their single-point closures at k*_-
    # (Tab. ccux_deg_one_col: X_M^- with weight sigma; Tab. num_deg_one: Q^{1,0}_{3,4})
    from fractions import Fraction
    for M, sig in ((1, Fraction(37, 100)), (2, Fraction(86, 100)), (3, Fraction(146, 100))):
        X, xi, Xb = BI.ccu_x(M, sig)
        out[f"X{M}_d1"] = _biased_entry(X, Xb, 2 * M + 2, 1, "Tab. ccux_deg_one_col")
    q, qc = BI.tuned_Q1034(mp.mpf(1))
    out["Q1034_1_d1"] = _biased_entry(q, qc, 6, 2, "Tab. num_deg_one (closure: the mirrored Q^{0,1}_{4,3})")
    return out


def _biased_entry(interior, closure, order, kc, cite):
    b = BI.to_biased(interior, closure, kc)
    return {"d": 1, "order": order, "biased": True, "a": b.a, "lo": b.lo, "rhs": list(b.rhs),
            "c_sup": b.c_sup, "c_lo": b.c_lo, "closure": list(b.closure), "kc": kc, "cite": cite}


if __name__ == "__main__":
    data = build()
    with open(os.path.join(HERE, "schemes.json"), "w") as fh:
        json.dump(data, fh, indent=1)
        fh.write("\n")
    print("wrote", len(data) - 1, "schemes")
