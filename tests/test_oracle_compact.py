"""Pins for the oracle's compact staggered operators (Sec. 3.1, Lele 1992 schemes).

* The interior coefficients are re-derived here from Taylor-matching conditions in exact
  rational arithmetic (not copied from the oracle).
* Every operator, with its boundary closures, is exact on polynomials of degree <= 4.
* Observed order: 6 in the interior, >= 4 globally.
"""
from fractions import Fraction

import numpy as np
import pytest
import sympy

from oracle import compact as C


def _solve_taylor(kind):
    al, a, b = sympy.symbols("alpha a b")
    eqs = []
    if kind == "D":
        # alpha (g'_{-1} + g'_{+1}) + g'_0 = a (f_{1/2} - f_{-1/2}) + b/3 (f_{3/2} - f_{-3/2})
        for k in (1, 3, 5):
            lhs = al * (k * (-1) ** (k - 1) + k) + (1 if k == 1 else 0)
            rhs = a * (sympy.Rational(1, 2) ** k - sympy.Rational(-1, 2) ** k) \
                + b / 3 * (sympy.Rational(3, 2) ** k - sympy.Rational(-3, 2) ** k)
            eqs.append(sympy.Eq(lhs, rhs))
    else:
        for k in (0, 2, 4):
            lhs = al * ((-1) ** k + 1) + (1 if k == 0 else 0)
            rhs = a / 2 * (sympy.Rational(1, 2) ** k + sympy.Rational(-1, 2) ** k) \
                + b / 2 * (sympy.Rational(3, 2) ** k + sympy.Rational(-3, 2) ** k)
            eqs.append(sympy.Eq(lhs, rhs))
    sol = sympy.solve(eqs, [al, a, b])
    return {k: Fraction(int(sympy.fraction(v)[0]), int(sympy.fraction(v)[1]))
            for k, v in zip(("alpha", "a", "b"), (sol[al], sol[a], sol[b]))}


def test_interior_coefficients_from_taylor_conditions():
    assert _solve_taylor("D") == C.DERIV6
    assert _solve_taylor("I") == C.INTERP6


@pytest.mark.parametrize("n", [8, 13, 40])
@pytest.mark.parametrize("deg", [0, 1, 2, 3, 4])
def test_polynomial_exactness(n, deg):
    xc = np.arange(n) + 0.5
    xf = np.arange(n + 1.0)
    s = float(n) ** deg + 1.0

    def f(x):
        return (x / 3.0 - 0.7) ** deg

    def df(x):
        return deg / 3.0 * (x / 3.0 - 0.7) ** (deg - 1) if deg else 0.0 * x

    tol = 1e-12 * max(1.0, (n / 3.0) ** deg)
    assert np.abs(C.icf(f(xc), 0) - f(xf)).max() < tol
    assert np.abs(C.dcf(f(xc), 0) - df(xf)).max() < tol
    assert np.abs(C.ifc(f(xf), 0) - f(xc)).max() < tol
    assert np.abs(C.dfc(f(xf), 0) - df(xc)).max() < tol
    w = float(f(np.array([0.0]))[0])
    assert np.abs(C.icf(f(xc), 0, wall_value=w) - f(xf)).max() < tol
    assert np.abs(C.dcf(f(xc), 0, wall_value=w) - df(xf)).max() < tol


def test_operators_act_along_any_axis():
    rng = np.random.default_rng(0)
    a = rng.standard_normal((7, 11))
    assert np.allclose(C.icf(a, 1), C.icf(a.T, 0).T, rtol=0, atol=1e-15)
    assert np.allclose(C.dfc(a, 0), C.dfc(a.T, 1).T, rtol=0, atol=1e-15)


def _errors(n, which):
    k, ph = 5.0, 0.3
    xc = (np.arange(n) + 0.5) / n
    xf = np.arange(n + 1.0) / n
    if which == "dcf":
        return C.dcf(np.sin(k * xc + ph), 0) * n - k * np.cos(k * xf + ph)
    if which == "icf":
        return C.icf(np.sin(k * xc + ph), 0) - np.sin(k * xf + ph)
    if which == "dfc":
        return C.dfc(np.sin(k * xf + ph), 0) * n - k * np.cos(k * xc + ph)
    return C.ifc(np.sin(k * xf + ph), 0) - np.sin(k * xc + ph)


@pytest.mark.parametrize("which", ["dcf", "icf", "dfc", "ifc"])
def test_convergence_orders(which):
    e1, e2 = _errors(64, which), _errors(128, which)
    glob = np.log2(np.abs(e1).max() / np.abs(e2).max())
    assert glob > 3.8
    # interior (middle half of the line): the boundary influence has decayed below rounding
    m1 = np.abs(e1[len(e1) // 4: 3 * len(e1) // 4]).max()
    m2 = np.abs(e2[len(e2) // 4: 3 * len(e2) // 4]).max()
    assert np.log2(m1 / m2) > 5.7
