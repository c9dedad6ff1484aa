"""Pins for the three-dimensional oracle (oracle/flow3d.py: spanwise-periodic direction, jet from
a circular orifice).

* Periodic compact operators: on a periodic line every Fourier mode is an eigenvector, and the
  interpolation and derivative multiply it by the closed-form transfer functions of the sixth-order
  staggered schemes, (a cos(t/2) + b cos(3t/2)) / (1 + 2 alpha cos t) and
  (2 a sin(t/2) + 2 b/3 sin(3t/2)) / (1 + 2 alpha cos t), with the half-cell phase shift.
* z-invariance: a state that does not depend on z, with w = 0 and no jet, gives in every z-plane
  the right-hand side of the two-dimensional oracle (pinned on its own), and R_w = 0.
* Mirror symmetry: a state symmetric about the jet's spanwise centre gives a right-hand side with
  the same symmetry (R_w odd), which a sign or index error in a z-term breaks.
* PDE consistency: on smooth manufactured fields periodic in z the discrete right-hand side of a
  perfect gas converges at the design order to the continuous one (sympy, Eqs. 1-6, 9, 10, 22, 24
  in three dimensions), away from the x and y boundary closures that the two-dimensional test
  pins.
* Jet boundary values: the sonic jet's state gives back the momentum ratio J and the pressure
  ratio J Ma^2; the Dirichlet mass flux of the wall faces is rho_j v_j at the orifice centre and
  vanishes away from it.
"""
import math

import numpy as np
import pytest
import sympy

from oracle import compact as C
from oracle import flow as F
from oracle import flow3d as F3
from paper_2210_05547_gb300 import inputs as I


@pytest.mark.parametrize("op,kind", [(C.icf_p, "I"), (C.ifc_p, "I"), (C.dcf_p, "D"),
                                     (C.dfc_p, "D")])
def test_periodic_operator_symbols(op, kind):
    n = 24
    a, b, al = (1.5, 0.1, 0.3) if kind == "I" else (63 / 62, 17 / 62, 9 / 62)
    cf = op in (C.icf_p, C.dcf_p)
    k = np.arange(n)
    for m in (1, 4, 7, 11):
        t = 2 * np.pi * m / n
        xin = k + 0.5 if cf else k            # centres, or faces
        xout = k if cf else k + 0.5
        f = np.exp(1j * t * xin)
        if kind == "I":
            sym = (a * np.cos(t / 2) + b * np.cos(1.5 * t)) / (1 + 2 * al * np.cos(t))
        else:
            sym = 1j * (2 * a * np.sin(t / 2) + 2 * b / 3 * np.sin(1.5 * t)) / (1 + 2 * al * np.cos(t))
        g = op(f.real, 0) + 1j * op(f.imag, 0)
        assert np.max(np.abs(g - sym * np.exp(1j * t * xout))) < 1e-13, m


def _nstate3(ns, nx, ny, nz):
    return sum(a * b * c for _, (a, b, c) in F3.state_layout(ns, nx, ny, nz))


def _extrude(U2, ns, nx, ny, nz):
    f = F.unpack(ns, nx, ny, U2)
    out = {k: np.broadcast_to(v, (nz,) + v.shape) for k, v in f.items()}
    out["rhow"] = np.zeros((nz, ny, nx))
    return F3.pack(ns, nx, ny, nz, out)


@pytest.mark.parametrize("maker", [lambda: I.bl_case(40, 24, seed=2), lambda: I.sbli_case(48, 24, seed=3)],
                         ids=["bl", "sbli"])
def test_z_uniform_state_gives_the_2d_rhs(table, maker):
    cfg2 = maker()
    nx, ny, nz = cfg2["nx"], cfg2["ny"], 6
    cfg3 = dict(cfg2, nz=nz, z0=0.0, z1=3.0, jet=0)
    case2 = F.make_case(cfg2, table, I.state_noise(sum(a * b for _, (a, b) in F.state_layout(5, nx, ny)), 2))
    case3 = F3.make_case(cfg3, table)
    case3.U_ref = _extrude(case2.U_ref, 5, nx, ny, nz)
    U3 = _extrude(case2.U0, 5, nx, ny, nz)
    R2 = F.unpack(5, nx, ny, F.rhs(case2, case2.U0))
    R3 = F3.unpack(5, nx, ny, nz, F3.rhs(case3, U3))
    for name, v2 in R2.items():
        scale = max(np.abs(v2).max(), 1e-300)
        for k in range(nz):
            assert np.abs(R3[name][k] - v2).max() <= 1e-12 * scale, (name, k)
    assert np.abs(R3["rhow"]).max() <= 1e-12 * np.abs(R3["rhou"]).max()


def test_mirror_symmetry_about_the_jet(table):
    cfg = I.jet_case(40, 24, 8, seed=4)
    cfg.update(jet_z=5.0, noise_amp=0.0)          # z = 5 is a z-face of the 8-cell periodic line
    case = F3.make_case(cfg, table)
    nx, ny, nz = 40, 24, 8
    R = F3.unpack(5, nx, ny, nz, F3.rhs(case, case.U0))
    # centres: z_k = (k + 1/2) dz mirror to 10 - z_k, i.e. k -> 7 - k; z-faces: k -> (8 - k) mod 8
    for name, v in R.items():
        scale = max(np.abs(v).max(), 1e-300)
        if name == "rhow":
            mirrored = -np.roll(v[::-1], 1, axis=0)
        else:
            mirrored = v[::-1]
        assert np.abs(v - mirrored).max() <= 1e-12 * scale, name
    assert np.abs(R["rhow"]).max() > 1e-6 * np.abs(R["rhov"]).max()      # the jet drives w


def test_jet_boundary_values(table):
    cfg = I.jet_case(256, 16, 128, seed=5)
    case = F3.make_case(cfg, table)
    mflux, T_j = F3.jet_state(cfg, case.sc)
    sc = case.sc
    rho_j = cfg["jet_J"] * sc.mach ** 2 * sc.p / (sc.R * T_j) / sc.rho
    v_j = mflux / rho_j
    assert abs(rho_j * v_j ** 2 / sc.mach ** 2 / cfg["jet_J"] - 1.0) < 1e-14
    assert abs(v_j ** 2 * sc.a ** 2 / (sc.gamma * sc.R * T_j) - 1.0) < 1e-14     # sonic
    f = F3.unpack(5, 256, 16, 128, case.U_ref)
    g = case.grid
    Xw, Zw = np.meshgrid(g.xc, case.zc)
    Lz = cfg["z1"] - cfg["z0"]
    dz = np.abs(Zw - cfg["jet_z"])
    r = np.hypot(Xw - cfg["jet_x"], np.minimum(dz, Lz - dz))
    wall = f["rhov"][:, 0, :]
    centre = r < 0.2 * cfg["jet_radius"]
    # the blend at the centre is 1 - O(exp(-2 / jet_edge)): within 2% of rho_j v_j
    assert centre.any() and np.allclose(wall[centre], mflux, rtol=2e-2, atol=0)
    assert np.all(np.abs(wall[r > 4.0 * cfg["jet_radius"]]) < 1e-8 * mflux)


# ------------------------------------------------------------------------------------------
# Manufactured fields periodic in z (calorically perfect gas)
# ------------------------------------------------------------------------------------------

def _mms3(cfg):
    x, y, z = sympy.symbols("x y z", real=True)
    Lx, Ly, Lz = cfg["x1"] - cfg["x0"], cfg["y1"] - cfg["y0"], cfg["z1"] - cfg["z0"]
    X = 2 * sympy.pi * (x - cfg["x0"]) / Lx
    Yv = 2 * sympy.pi * (y - cfg["y0"]) / Ly
    Z = 2 * sympy.pi * (z - cfg["z0"]) / Lz
    r = sympy.Rational
    rho = 1 + r(2, 10) * sympy.sin(X + r(1, 10)) * sympy.cos(Yv + r(2, 10)) + r(1, 10) * sympy.cos(Z)
    u = r(3, 2) + r(3, 10) * sympy.cos(X) * sympy.sin(Yv + r(1, 2)) * sympy.cos(Z + r(1, 5))
    v = r(2, 10) * sympy.sin(X + 1) * sympy.cos(Yv) + r(1, 10) * sympy.sin(Z)
    w = r(2, 10) * sympy.cos(X + r(1, 3)) * sympy.sin(Yv) + r(3, 10) * sympy.sin(Z + r(1, 4))
    Tf = 1 + r(2, 10) * sympy.cos(X + r(3, 10)) * sympy.cos(Yv + r(1, 10)) * sympy.cos(Z + r(1, 2))
    return (x, y, z), rho, u, v, w, Tf


def _exact3(cfg, sc):
    (x, y, z), rho, u, v, w, Tshape = _mms3(cfg)
    g = sc.gamma
    T = Tshape / (g - 1)
    p = rho * (g - 1) / g * T
    mu = F.SUTHERLAND_C1 * (T * sc.T_ref) ** sympy.Rational(3, 2) / (T * sc.T_ref + F.SUTHERLAND_TS) / sc.mu
    Re, Pr = sc.Re, sc.Pr
    vel = (u, v, w)
    X = (x, y, z)
    grad = [[sympy.diff(vel[i], X[j]) for j in range(3)] for i in range(3)]
    div = grad[0][0] + grad[1][1] + grad[2][2]
    tau = [[mu / Re * (grad[i][j] + grad[j][i] - (sympy.Rational(2, 3) * div if i == j else 0))
            for j in range(3)] for i in range(3)]
    q = [-mu / (Re * Pr) * sympy.diff(T, X[j]) for j in range(3)]
    E = T / g + (u * u + v * v + w * w) / 2
    H = E + p / rho
    R = {"rho": -sum(sympy.diff(rho * vel[j], X[j]) for j in range(3))}
    for i, name in enumerate(("rhou", "rhov", "rhow")):
        R[name] = -sum(sympy.diff(rho * vel[i] * vel[j] + (p if i == j else 0) - tau[i][j], X[j])
                       for j in range(3))
    R["rhoE"] = -sum(sympy.diff(rho * H * vel[j] + q[j] - sum(tau[j][i] * vel[i] for i in range(3)),
                                X[j]) for j in range(3))
    prim = dict(rho=rho, u=u, v=v, w=w, E=E)
    return {k: sympy.lambdify((x, y, z), val, "numpy")
            for k, val in {**R, **{"p_" + k: val for k, val in prim.items()}}.items()}


def _mms_case(nx, ny, nz):
    cfg = I.box_case(nx, ny, kind="cpg")
    cfg.update(x0=0.0, x1=1.3, y0=0.0, y1=1.0, y_stretch="tanh", y_param=1.2, reynolds=50.0,
               sponge_in=0.0, sponge_out=0.0, sponge_top_cells=0, mach=1.5, nz=nz, z0=0.0,
               z1=0.9, jet=0)
    return cfg


def test_pde_consistency_3d_perfect_gas(table):
    errs = []
    for nx, ny, nz in ((14, 12, 10), (28, 24, 20), (56, 48, 40)):
        cfg = _mms_case(nx, ny, nz)
        case = F3.make_case(cfg, table)
        f = _exact3(cfg, case.sc)
        g = case.grid
        zc, zf = case.zc, case.zf
        nodes = {"c": (g.xc, g.yc, zc), "xf": (g.xf, g.yc, zc), "yf": (g.xc, g.yf, zc),
                 "zf": (g.xc, g.yc, zf)}

        def at(node, key):
            xs, ys, zs = nodes[node]
            Z3, Y3, X3 = np.meshgrid(zs, ys, xs, indexing="ij")
            return np.broadcast_to(f[key](X3, Y3, Z3), Z3.shape)

        fields = {"rho": at("c", "p_rho"), "rhoE": at("c", "p_rho") * at("c", "p_E"),
                  "rhou": at("xf", "p_rho") * at("xf", "p_u"),
                  "rhov": at("yf", "p_rho") * at("yf", "p_v"),
                  "rhow": at("zf", "p_rho") * at("zf", "p_w")}
        fields["rs1"] = 0.233 * fields["rho"]
        for s in range(2, 5):
            fields[f"rs{s}"] = 0.0 * fields["rho"]
        R = F3.unpack(5, nx, ny, nz, F3.rhs(case, F3.pack(5, nx, ny, nz, fields)))
        e = {}
        # the x and y boundary closures are pinned by the two-dimensional test; here the points
        # at least three cells from the x and y ends, where every z-term acts
        inner = (slice(None), slice(3, -3), slice(3, -3))
        for name, node in (("rho", "c"), ("rhoE", "c"), ("rhou", "xf"), ("rhov", "yf"),
                           ("rhow", "zf")):
            ex = at(node, name)
            d = (R[name] - ex)[inner]
            e[name] = np.abs(d).max() / np.abs(ex[inner]).max()
        errs.append(e)
    for name in errs[0]:
        order = math.log2(errs[1][name] / errs[2][name])
        assert errs[2][name] < 5e-3, (name, errs)
        assert order > 2.8, (name, [x[name] for x in errs])
