"""Pins for the oracle's thermally perfect gas (Eqs. 22-25): the heat capacity of Eq. (23) in its
harmonic-oscillator reading, Sutherland viscosity, Keyes conductivity.

* Printed constants: Theta and the Keyes coefficients equal the paper's values.
* c_p is the temperature derivative of the enthalpy the oracle integrates in closed form, and
  c_p(T_inf) = c_p,inf; its limits are c_p0 (vibration frozen) and c_p0 (1 + (gamma-1)/gamma)
  (vibration fully excited); with Theta -> infinity the energy is the calorically perfect one.
* The Newton inversion of e(T) round-trips over 50-20000 K.
* Keyes' law gives the handbook conductivity of air at 300 K (0.026 W/(m K)).
* PDE consistency: on smooth manufactured fields at a temperature where vibration matters the
  discrete right-hand side of the "tpg" kind converges to the continuous one built symbolically
  from Eqs. (1)-(6), (9), (10), (22)-(25) (a wrong energy or conductivity law fails it).
"""
import math

import numpy as np
import pytest
import sympy

from conftest import read_golden
from oracle import flow as F
from paper_2210_05547_gb300 import inputs as I
from test_oracle_flow import _errors_against, _mms_box, _mms_fields, _set_state_cpg


@pytest.fixture(scope="module")
def sc(table):
    return F.freestream_scales(table, "tpg", I.bl_case(kind="tpg"))


def test_printed_constants():
    g = read_golden("paper_constants.txt")
    assert F.TPG_THETA == g["tpg_theta"]
    assert (F.KEYES_C2, F.KEYES_C3, F.KEYES_C4) == (g["keyes_C2"], g["keyes_C3"], g["keyes_C4"])


def test_cp_is_derivative_of_enthalpy_and_matches_freestream(sc):
    T = np.geomspace(100.0, 20000.0, 57)
    h = lambda t: F.tpg_energy(sc, t) + sc.R * t
    d = 1e-5 * T
    num = (h(T + d) - h(T - d)) / (2 * d)
    assert np.max(np.abs(num / F.tpg_cp(sc, T) - 1.0)) < 1e-8
    assert abs(F.tpg_cp(sc, np.array(sc.T)) / sc.cp - 1.0) < 1e-15


def test_cp_limits_and_calorically_perfect_limit(sc, monkeypatch):
    cp0 = F.tpg_cp0(sc)
    assert abs(F.tpg_cp(sc, np.array(50.0)) / cp0 - 1.0) < 1e-20 + 1e-15
    hi = cp0 * (1.0 + (sc.gamma - 1.0) / sc.gamma)
    assert abs(F.tpg_cp(sc, np.array(1e7)) / hi - 1.0) < 1e-6
    monkeypatch.setattr(F, "TPG_THETA", 1e9)
    T = np.array([300.0, 1000.0, 5000.0])
    assert np.allclose(F.tpg_energy(sc, T), (sc.cp - sc.R) * T, rtol=1e-14, atol=0)


def test_newton_round_trip(sc):
    T = np.geomspace(50.0, 20000.0, 301)
    e = F.tpg_energy(sc, T)
    assert np.max(np.abs(F.tpg_temperature(sc, e) / T - 1.0)) < 1e-13


def test_keyes_handbook_air():
    assert abs(float(F.keyes(300.0)) - 0.0263) < 0.02 * 0.0263


def _tpg_exact_rhs(cfg, sc):
    x, y, rho, u, v, Tshape = _mms_fields(cfg)
    g = sc.gamma
    T = Tshape / (g - 1)                               # nondimensional, freestream 1/(gamma - 1)
    Ts = T * sc.T_ref                                  # kelvin
    p = rho * (g - 1) / g * T                          # Eq. (22)
    cp0, th, g1 = F.tpg_cp0(sc), F.TPG_THETA, (g - 1) / g
    e = (cp0 * (Ts + g1 * th / (sympy.exp(th / Ts) - 1)) - sc.R * Ts) / sc.a ** 2
    mu = F.SUTHERLAND_C1 * Ts ** sympy.Rational(3, 2) / (Ts + F.SUTHERLAND_TS) / sc.mu
    k = F.KEYES_C2 * sympy.sqrt(Ts) / (1 + (F.KEYES_C3 / Ts) * 10 ** (-F.KEYES_C4 / Ts)) / sc.k
    Re, Pr = sc.Re, sc.Pr
    ux, uy, vx, vy = sympy.diff(u, x), sympy.diff(u, y), sympy.diff(v, x), sympy.diff(v, y)
    div = ux + vy
    txx = mu / Re * (2 * ux - sympy.Rational(2, 3) * div)
    tyy = mu / Re * (2 * vy - sympy.Rational(2, 3) * div)
    txy = mu / Re * (uy + vx)
    qx = -k / (Re * Pr) * sympy.diff(T, x)
    qy = -k / (Re * Pr) * sympy.diff(T, y)
    E = e + (u * u + v * v) / 2
    H = E + p / rho
    R = dict(
        rho=-(sympy.diff(rho * u, x) + sympy.diff(rho * v, y)),
        rhou=-(sympy.diff(rho * u * u + p - txx, x) + sympy.diff(rho * u * v - txy, y)),
        rhov=-(sympy.diff(rho * u * v - txy, x) + sympy.diff(rho * v * v + p - tyy, y)),
        rhoE=-(sympy.diff(rho * H * u + qx - (txx * u + txy * v), x)
               + sympy.diff(rho * H * v + qy - (txy * u + tyy * v), y)),
    )
    prim = dict(rho=rho, u=u, v=v, T=T, E=E)
    return {k: sympy.lambdify((x, y), val, "numpy")
            for k, val in {**R, **{"p_" + k: w for k, w in prim.items()}}.items()}


def test_pde_consistency_tpg(table):
    errs = []
    for nx, ny in ((26, 20), (52, 40), (104, 80)):
        cfg = _mms_box(nx, ny, "tpg")
        cfg["T_inf"] = 1500.0                          # Theta / T ~ 2: vibration half excited
        case = F.make_case(cfg, table)
        f = _tpg_exact_rhs(cfg, case.sc)
        U = _set_state_cpg(case, f)
        errs.append(_errors_against(case, U, f))
    for name in errs[0]:
        order = math.log2(errs[1][name] / errs[2][name])
        assert errs[2][name] < 2e-3, (name, errs)
        assert order > 2.8, (name, [e[name] for e in errs])
