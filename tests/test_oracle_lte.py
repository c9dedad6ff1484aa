"""Pins for the oracle's closure in local thermodynamic equilibrium (Sec. 2.2.2, special cases:
the composition is the one of minimum Gibbs energy, a function of the thermodynamic state).

* The composition at the returned (T, p) is the Gibbs minimum found at (T, p) by the bisection
  element-potential solve of the kinetics pins (itself pinned by brute-force search), over
  2500-14000 K and 1e-4-1 kg/m^3; element content and mass fractions are those of the air.
* Detailed balance: every reaction's net rate vanishes at that composition, so the equilibrium
  agrees with the equilibrium constants of the kinetics.
* The closed constant-(rho, e) reactor of finite-rate chemistry relaxes to the LTE state of the
  same (rho, e).
* c_v,eq is the central difference of the equilibrium energy at fixed rho; (dX_s/dT)_p is the
  central difference of the independent (T, p) equilibrium.
* Reactive conductivity: with one diffusion coefficient D for every species the algebraic
  diffusion of Eq. (18) is Fick's law in mass fractions, so k_reactive = rho D (c_p,eq - c_p,f)
  with c_p,eq the central difference of the equilibrium enthalpy at fixed p (independent solve).
* Cold limit: at 300-450 K the composition is the air itself (NO below 1e-10) and T the frozen
  inversion.
* The inversion e -> T round-trips over 300-20000 K.
"""
import numpy as np
import pytest
import scipy.integrate

from oracle import gas as G
from test_oracle_kinetics import gibbs_equilibrium

Y_AIR = np.array([0.767, 0.233, 0.0, 0.0, 0.0])


@pytest.fixture(scope="module")
def bm(table):
    return G.element_content(table, Y_AIR)


def _grid():
    T = np.array([2500.0, 4000.0, 6000.0, 9000.0, 14000.0])
    rho = np.array([1e-4, 1e-2, 1.0])
    TT, RR = np.meshgrid(T, rho)
    return TT.ravel(), RR.ravel()


def _lte_at(table, T, rho, bm):
    _, e, _, _ = G.equilibrium_at(table, T, rho, bm)
    return G.lte_eval(table, rho, e, bm)


def test_composition_is_the_gibbs_minimum(table, bm):
    T, rho = _grid()
    r = _lte_at(table, T, rho, bm)
    assert not r["status"].any()
    assert np.max(np.abs(r["T"] / T - 1.0)) < 1e-13
    for i in range(T.size):
        n = gibbs_equilibrium(table, r["T"][i], r["p"][i], bm)
        X_ref = n / n.sum()
        assert np.allclose(r["X"][:, i], X_ref, rtol=1e-9, atol=1e-13 * X_ref.max()), i
    assert np.allclose(r["Y"].sum(axis=0), 1.0, rtol=0, atol=1e-14)
    # frozen transport of that composition: the finite-rate closure's at the same state
    fz = G.thermo_eval(table, rho, G.mixture_energy(table, r["T"], r["Y"]), r["Y"])
    for key, ref in (("mu", "mu"), ("k_frozen", "k"), ("p", "p"), ("D", "D")):
        assert np.allclose(r[key], fz[ref], rtol=1e-12, atol=0), key
    assert np.allclose(G.element_content(table, r["Y"]), bm[:, None], rtol=1e-14, atol=0)


def test_detailed_balance(table, bm):
    T, rho = _grid()
    r = _lte_at(table, T, rho, bm)
    conc = rho * r["Y"] / table.M()[:, None]
    kf, _, R = G.reaction_rates(table, r["T"], conc)
    for ir, rx in enumerate(table.reactions):
        fwd = kf[ir] * np.prod(conc ** rx.nu_f[:, None], axis=0)
        assert np.all(np.abs(R[ir]) <= 1e-9 * fwd), ir


def test_closed_reactor_relaxes_to_the_lte_state(table, bm):
    rho = 0.05
    e = G.mixture_energy(table, np.array([6000.0]), Y_AIR[:, None])[0]

    def f(t, y):
        Y = y[:, None] / rho
        T, _ = G.temperature_from_energy(table, np.array([e]), Y)
        return G.production_rates(table, T, np.array([rho]), Y)[:, 0]

    sol = scipy.integrate.solve_ivp(f, (0.0, 1.0), rho * Y_AIR, method="Radau", rtol=1e-10,
                                    atol=1e-14)
    Yf = sol.y[:, -1] / rho
    Tf, _ = G.temperature_from_energy(table, np.array([e]), Yf[:, None])
    r = G.lte_eval(table, np.array([rho]), np.array([e]), bm)
    assert abs(r["T"][0] / Tf[0] - 1.0) < 1e-6
    assert np.allclose(r["Y"][:, 0], Yf, rtol=1e-5, atol=1e-9)


def test_equilibrium_heat_capacity(table, bm):
    T, rho = _grid()
    _, _, cv_eq, _ = G.equilibrium_at(table, T, rho, bm)
    d = 1e-4 * T
    _, ep, _, _ = G.equilibrium_at(table, T + d, rho, bm)
    _, em, _, _ = G.equilibrium_at(table, T - d, rho, bm)
    assert np.max(np.abs((ep - em) / (2 * d) / cv_eq - 1.0)) < 1e-6


def _x_eq(table, T, p, bm):
    n = gibbs_equilibrium(table, T, p, bm)
    return n / n.sum()


def test_mole_fraction_derivative_at_fixed_pressure(table, bm):
    T, rho = _grid()
    r = _lte_at(table, T, rho, bm)
    for i in range(T.size):
        Ti, pi = r["T"][i], r["p"][i]
        d = 1e-4 * Ti
        fd = (_x_eq(table, Ti + d, pi, bm) - _x_eq(table, Ti - d, pi, bm)) / (2 * d)
        scale = np.abs(fd).max()
        assert np.max(np.abs(r["dXdT"][:, i] - fd)) < 1e-6 * scale, i


def test_reactive_conductivity_for_equal_diffusivities(table, bm, monkeypatch):
    D = 3.0e-4
    monkeypatch.setattr(G, "averaged_diffusion", lambda tab, X, Dbin: np.full_like(X, D))
    T, rho = _grid()
    r = _lte_at(table, T, rho, bm)
    M = table.M()
    for i in range(T.size):
        Ti, pi = r["T"][i], r["p"][i]
        d = 1e-4 * Ti

        def h_eq(t):
            X = _x_eq(table, t, pi, bm)
            H = np.array([G.species_molar_enthalpy(s, np.array([t]))[0] for s in table.species])
            return (X @ H) / (X @ M)

        cp_eq = (h_eq(Ti + d) - h_eq(Ti - d)) / (2 * d)
        cp_f = r["cv"][i] + r["R"][i]
        expect = rho[i] * D * (cp_eq - cp_f)
        assert abs(r["k_reactive"][i] - expect) < 1e-6 * abs(expect) + 1e-12 * r["k_frozen"][i], i
        assert r["k_reactive"][i] > 0.0
        # the conductivity the heat flux uses is the frozen one plus that reactive part
        assert abs(r["k"][i] - (r["k_frozen"][i] + expect)) < 1e-6 * r["k"][i], i


def test_cold_limit_is_frozen_air(table, bm):
    T = np.array([300.0, 380.0, 450.0])
    rho = np.array([0.01, 0.1, 1.0])
    r = _lte_at(table, T, rho, bm)
    assert np.allclose(r["Y"], Y_AIR[:, None], rtol=0, atol=1e-10)
    e = G.mixture_energy(table, T, np.repeat(Y_AIR[:, None], 3, axis=1))
    Tf, _ = G.temperature_from_energy(table, e, np.repeat(Y_AIR[:, None], 3, axis=1))
    assert np.allclose(r["T"], Tf, rtol=1e-9)
    assert np.all(np.abs(r["k_reactive"]) < 1e-6 * r["k_frozen"])


def test_round_trip(table, bm):
    T = np.geomspace(300.0, 20000.0, 41)
    rho = np.geomspace(1e-4, 1.0, 41)[::-1]
    _, e, _, _ = G.equilibrium_at(table, T, rho, bm)
    r = G.lte_eval(table, rho, e, bm)
    assert not r["status"].any()
    assert np.max(np.abs(r["T"] / T - 1.0)) < 1e-13


# ------------------------------------------------------------------------------------------
# The right-hand side with the LTE closure
# ------------------------------------------------------------------------------------------

def test_freestream_preservation_lte(table):
    from oracle import flow as F
    from paper_2210_05547_gb300 import inputs as I
    cfg = I.box_case(24, 16, kind="lte")
    case = F.make_case(cfg, table)
    parts = F.unpack(5, 24, 16, F.rhs(case, case.U0))
    ref = F.unpack(5, 24, 16, case.U0)
    for name in parts:
        assert np.abs(parts[name]).max() < 1e-13 * max(np.abs(ref[name]).max(), 1.0), name


def test_cold_lte_right_hand_side_is_the_frozen_one(table):
    """At 240-360 K the equilibrium holds the air's composition (NO below 1e-14), so the LTE and
    frozen-chemistry right-hand sides of one state agree to rounding (1e-10 of max|R|: the right-hand
    side is a small difference of the fluxes)."""
    from oracle import flow as F
    from test_oracle_flow import _mms_box, _mms_fields, _nodes
    import sympy
    out = {}
    for kind in ("lte", "frozen"):
        cfg = _mms_box(40, 32, kind)
        cfg["T_inf"] = 300.0
        case = F.make_case(cfg, table)
        sc, g = case.sc, case.grid
        x, y, rho_e, u_e, v_e, T_e = _mms_fields(cfg)
        f = {k: sympy.lambdify((x, y), val, "numpy")
             for k, val in dict(rho=rho_e, u=u_e, v=v_e, T=300 * T_e).items()}
        nd = _nodes(g)
        Xc, Yc = nd["c"]
        rho = f["rho"](Xc, Yc)
        air = np.repeat(Y_AIR[:, None], rho.size, axis=1)
        e = G.mixture_energy(table, f["T"](Xc, Yc).ravel(), air).reshape(rho.shape) / sc.a ** 2
        Xu, Yu = nd["xf"]
        Xv, Yv = nd["yf"]
        uc = f["u"](Xc, Yc)
        vc = f["v"](Xc, Yc)
        fields = {"rho": rho, "rhoE": rho * (e + 0.5 * (uc * uc + vc * vc)),
                  "rhou": f["rho"](Xu, Yu) * f["u"](Xu, Yu), "rhov": f["rho"](Xv, Yv) * f["v"](Xv, Yv)}
        for s in range(1, 5):
            fields[f"rs{s}"] = Y_AIR[s] * rho
        out[kind] = F.unpack(5, 40, 32, F.rhs(case, F.pack(5, 40, 32, fields)))
    for name in ("rho", "rhou", "rhov", "rhoE"):
        a, b = out["lte"][name], out["frozen"][name]
        assert np.abs(a - b).max() <= 1e-10 * np.abs(b).max(), name


def _lte_reference(cfg, case, bm):
    """Continuous right-hand side of the LTE model on the manufactured fields: pointwise LTE
    closure calls at the exact density and temperature, fluxes of Eqs. (5), (6), (9) and the
    heat flux -k_eq grad T, and fourth-order central differences of those fluxes."""
    import sympy
    from test_oracle_flow import _mms_fields
    sc, tab = case.sc, case.tab
    x, y, rho_e, u_e, v_e, T_e = _mms_fields(cfg)
    Tsi_e = cfg["T_inf"] * T_e
    prim = {k: sympy.lambdify((x, y), val, "numpy")
            for k, val in dict(rho=rho_e, u=u_e, v=v_e, Tsi=Tsi_e).items()}
    grads = {k + d: sympy.lambdify((x, y), sympy.diff(val, sym), "numpy")
             for k, val in dict(u=u_e, v=v_e, Tsi=Tsi_e).items() for d, sym in (("x", x), ("y", y))}

    def fluxes(X, Yy):
        X = np.atleast_1d(X).astype(float)
        Yy = np.broadcast_to(np.atleast_1d(Yy).astype(float), X.shape)
        one = np.ones(X.size)
        rho = prim["rho"](X, Yy) * one
        Tsi = prim["Tsi"](X, Yy) * one
        u = prim["u"](X, Yy) * one
        v = prim["v"](X, Yy) * one
        _, e_si, _, _ = G.equilibrium_at(tab, Tsi, rho * sc.rho, bm)
        th = G.lte_eval(tab, rho * sc.rho, e_si, bm)
        p = th["p"] / (sc.rho * sc.a ** 2)
        mu, k = th["mu"] / sc.mu, th["k"] / sc.k
        Re, Pr = sc.Re, sc.Pr
        ux, uy = grads["ux"](X, Yy), grads["uy"](X, Yy)
        vx, vy = grads["vx"](X, Yy), grads["vy"](X, Yy)
        Tx, Ty = grads["Tsix"](X, Yy) / sc.T_ref, grads["Tsiy"](X, Yy) / sc.T_ref
        div = ux + vy
        txx = mu / Re * (2 * ux - 2 / 3 * div)
        tyy = mu / Re * (2 * vy - 2 / 3 * div)
        txy = mu / Re * (uy + vx)
        E = e_si / sc.a ** 2 + 0.5 * (u * u + v * v)
        H = E + p / rho
        Fx = dict(rho=rho * u, rhou=rho * u * u + p - txx, rhov=rho * u * v - txy,
                  rhoE=rho * H * u - k / (Re * Pr) * Tx - (txx * u + txy * v))
        Fy = dict(rho=rho * v, rhou=rho * u * v - txy, rhov=rho * v * v + p - tyy,
                  rhoE=rho * H * v - k / (Re * Pr) * Ty - (txy * u + tyy * v))
        return Fx, Fy, (rho, u, v, E)

    def exact(X, Yy):
        h = 1e-4
        fx = [fluxes(X + s * h, Yy)[0] for s in (1, -1, 2, -2)]
        fy = [fluxes(X, Yy + s * h)[1] for s in (1, -1, 2, -2)]
        out = {}
        for name in fx[0]:
            dFx = (8 * (fx[0][name] - fx[1][name]) - (fx[2][name] - fx[3][name])) / (12 * h)
            dFy = (8 * (fy[0][name] - fy[1][name]) - (fy[2][name] - fy[3][name])) / (12 * h)
            out[name] = -(dFx + dFy)
        return out

    return fluxes, exact


def test_pde_consistency_lte_dissociating(table, bm):
    """Manufactured fields at 3200-4800 K and 0.1 bar, where oxygen dissociates and the reactive
    conductivity exceeds the frozen one: the discrete right-hand side converges to the continuous
    one at the design order (a wrong equilibrium pressure, energy or conductivity fails it)."""
    import math
    from oracle import flow as F
    from test_oracle_flow import _mms_box, _nodes
    errs = []
    for nx, ny in ((26, 20), (52, 40), (104, 80)):
        cfg = _mms_box(nx, ny, "lte")
        cfg.update(T_inf=4000.0, p_inf=1.0e4)
        case = F.make_case(cfg, table)
        fluxes, exact = _lte_reference(cfg, case, bm)
        g = case.grid
        nd = _nodes(g)
        Xc, Yc = nd["c"]
        _, _, (rho, _, _, E) = fluxes(Xc.ravel(), Yc.ravel())
        fields = {"rho": rho.reshape(Xc.shape), "rhoE": (rho * E).reshape(Xc.shape)}
        fields["rs1"] = 0.233 * fields["rho"]
        for s in range(2, 5):
            fields[f"rs{s}"] = 0.0 * Xc
        Xu, Yu = nd["xf"]
        _, _, (r, u, _, _) = fluxes(Xu.ravel(), Yu.ravel())
        fields["rhou"] = (r * u).reshape(Xu.shape)
        Xv, Yv = nd["yf"]
        _, _, (r, _, v, _) = fluxes(Xv.ravel(), Yv.ravel())
        fields["rhov"] = (r * v).reshape(Xv.shape)
        R = F.unpack(5, g.nx, g.ny, F.rhs(case, F.pack(5, g.nx, g.ny, fields)))
        e = {}
        for name, node in (("rho", "c"), ("rhoE", "c"), ("rhou", "xf"), ("rhov", "yf")):
            Xn, Yn = nd[node]
            ex = exact(Xn.ravel(), Yn.ravel())[name].reshape(Xn.shape)
            d = R[name] - ex
            if name == "rhou":
                d, ex = d[:, 1:-1], ex[:, 1:-1]
            if name == "rhov":
                d, ex = d[1:-1, :], ex[1:-1, :]
            e[name] = np.abs(d).max() / np.abs(ex).max()
        errs.append(e)
    for name in errs[0]:
        order = math.log2(errs[1][name] / errs[2][name])
        assert errs[2][name] < 5e-3, (name, errs)
        assert order > 2.8, (name, [x[name] for x in errs])
