"""FP64 oracle: three-dimensional right-hand side with a spanwise-periodic direction and a jet
issuing from the wall (the sonic jet in hypersonic crossflow of Sec. 4, here with a circular
orifice on a spanwise-periodic domain).

TEST INFRASTRUCTURE (see oracle/gas.py header). Not used by the product path.

The paper's jet case is two-dimensional (a slot); its equations, closure and discretisation are
those of the two-dimensional oracle (oracle/flow.py) with the third direction added:

* arrays indexed [k, j, i] (z, y, x), x fastest; centres (nz, ny, nx) hold rho, rho_s (all but
  the first species), rho E; rho u on x-faces (nz, ny, nx+1), rho v on y-faces (nz, ny+1, nx),
  rho w on z-faces (nz, ny, nx; face k lies between centres k-1 and k, periodic);
* z is uniform and periodic: the compact operators of oracle/compact.py with every row interior
  and indices modulo nz;
* shear stresses and cross momentum fluxes live on the edges of their plane: tau_xy on xy-edges
  (nz, ny+1, nx+1), tau_xz on xz-edges (nz, ny, nx+1), tau_yz on yz-edges (nz, ny+1, nx);
* the artificial diffusivities take fourth differences and the Gaussian filter in z as well
  (periodic there), with the three-dimensional strain and vorticity;
* the jet (reading; the paper gives a sonic jet of prescribed pressure and temperature ratios and
  momentum ratio J): inside a circular orifice of radius r_j centred at (x_j, z_j) the wall face
  holds the Dirichlet mass flux rho_j v_j of a sonic jet at T_j = T_jet_ratio T_inf with
  p_j = J Ma_inf^2 p_inf (so that J = rho_j v_j^2 / (rho_inf U_inf^2)), blended to the no-slip
  wall by a tanh of width jet_edge r_j; the wall temperature of the heat flux blends from T_wall
  to T_j the same way; u = w = 0 and no diffusion through the wall. The reference and initial
  states carry the jet's plume, so that the first cells above the orifice hold its density and
  momentum: the two-dimensional profile's T, p, u, v are blended towards (T_j, p_j, 0, v_j) with
  F = f(r) exp(-((y - y0) / (2 r_j))^2), and the wall faces hold rho v of that blend.

Every step follows the two-dimensional sequence of oracle.flow.rhs; with a z-uniform state and no
jet each z-plane gives exactly that right-hand side (pinned in tests/test_oracle_flow3d.py).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import compact as C
from . import flow as F
from . import gas as G


@dataclasses.dataclass
class Case3D:
    cfg: dict
    tab: G.GasTable
    kind: str
    sc: F.Scales
    grid: F.Grid
    nz: int
    zeta: float           # d(zeta)/dz, uniform
    zc: np.ndarray        # z of the centres (and of the x- and y-faces)
    zf: np.ndarray        # z of the z-faces
    U_ref: np.ndarray
    sigma: dict           # sponge strength at 'c', 'xf', 'yf', 'zf'
    U0: np.ndarray
    jet: np.ndarray       # (nz, nx) blend factor of the orifice at the wall faces
    T_wall_face: np.ndarray   # (nz, nx) wall temperature of the heat flux, K


def state_layout(ns, nx, ny, nz):
    out = [("rho", (nz, ny, nx))]
    out += [(f"rs{s}", (nz, ny, nx)) for s in range(1, ns)]
    out += [("rhoE", (nz, ny, nx)), ("rhou", (nz, ny, nx + 1)), ("rhov", (nz, ny + 1, nx)),
            ("rhow", (nz, ny, nx))]
    return out


def pack(ns, nx, ny, nz, fields):
    return np.concatenate([np.asarray(fields[name], dtype=np.float64).ravel()
                           for name, _ in state_layout(ns, nx, ny, nz)])


def unpack(ns, nx, ny, nz, U):
    out, off = {}, 0
    for name, shape in state_layout(ns, nx, ny, nz):
        size = shape[0] * shape[1] * shape[2]
        out[name] = np.asarray(U[off:off + size]).reshape(shape)
        off += size
    assert off == U.size
    return out


def jet_blend(cfg, x, z):
    """Orifice blend factor at wall points (x, z): 1/2 (1 - tanh((r - r_j) / (edge r_j))) with r the
    distance to the jet centre, the spanwise separation taken on the periodic domain."""
    Lz = cfg["z1"] - cfg["z0"]
    dz = np.abs(z - cfg["jet_z"])
    dz = np.minimum(dz, Lz - dz)
    r = np.sqrt((x - cfg["jet_x"]) ** 2 + dz ** 2)
    rj = cfg["jet_radius"]
    return 0.5 * (1.0 - np.tanh((r - rj) / (cfg["jet_edge"] * rj)))


def jet_state(cfg, sc):
    """Nondimensional mass flux rho_j v_j and the jet temperature (K) of the sonic jet."""
    T_j, p_j, v_j = jet_primitives(cfg, sc)
    rho_j = p_j / (sc.R * T_j) / sc.rho
    return rho_j * v_j, T_j


def jet_primitives(cfg, sc):
    """T_j (K), p_j (Pa) and the nondimensional v_j of the sonic jet."""
    T_j = cfg["jet_T_ratio"] * sc.T
    p_j = cfg["jet_J"] * sc.mach ** 2 * sc.p
    v_j = math.sqrt(sc.gamma * sc.R * T_j) / sc.a
    return T_j, p_j, v_j


JET_PLUME_HEIGHT = 2.0       # plume height of the initial state, in orifice radii


def plume(cfg, x, y, z):
    """Blend factor of the jet's plume at (x, y, z)."""
    h = JET_PLUME_HEIGHT * cfg["jet_radius"]
    return jet_blend(cfg, x, z) * np.exp(-((y - cfg["y0"]) / h) ** 2)


def make_case(cfg, tab, noise=None) -> Case3D:
    """Reference and initial states: the two-dimensional profile of oracle.flow at every z, the
    jet's mass flux on the wall faces of the orifice; noise as in two dimensions (none on the
    Dirichlet boundary faces)."""
    kind = cfg["kind"]
    if kind not in (F.KIND_CNEQ, F.KIND_FROZEN, F.KIND_CPG, F.KIND_TPG):
        raise ValueError("three-dimensional cases take the cneq, frozen, cpg or tpg gas")
    sc = F.freestream_scales(tab, kind, cfg)
    g = F.make_grid(cfg)
    nx, ny, nz, ns = g.nx, g.ny, cfg["nz"], tab.ns
    dz = (cfg["z1"] - cfg["z0"]) / nz
    zf = cfg["z0"] + dz * np.arange(nz)
    zc = zf + 0.5 * dz
    ref = {}
    jet_on = bool(cfg.get("jet", 0))
    if jet_on:
        T_j, p_j, v_j = jet_primitives(cfg, sc)

    def nodes(xs, ys):
        """Conserved rho, rho_s, rho E and the velocities at (z, y, x) nodes with the plume."""
        Zn, Yn, Xn = np.meshgrid(zc, ys, xs, indexing="ij")
        T, p, u, v, Y = F._primitive_profile(cfg, sc, tab, kind, Xn[0], Yn[0])
        T, p, u, v = (np.broadcast_to(a, Zn.shape) for a in (T, p, u, v))
        Y = np.broadcast_to(Y[:, None], (tab.ns,) + Zn.shape)
        if jet_on:
            Fp = plume(cfg, Xn, Yn, Zn)
            T = T + (T_j - T) * Fp
            p = p + (p_j - p) * Fp
            u = u * (1.0 - Fp)
            v = v + (v_j - v) * Fp
        rho, rhoY, rhoE = F._conserved_from_primitive(tab, kind, sc, np.array(T), np.array(p),
                                                      np.array(u), np.array(v), np.array(Y))
        return rho, rhoY, rhoE, u, v

    rho, rhoY, rhoE, _, _ = nodes(g.xc, g.yc)
    ref["rho"] = rho
    for s in range(1, ns):
        ref[f"rs{s}"] = rhoY[s]
    ref["rhoE"] = rhoE
    rho_u, _, _, u, _ = nodes(g.xf, g.yc)
    ref["rhou"] = rho_u * u
    rho_v, _, _, _, v = nodes(g.xc, g.yf)
    ref["rhov"] = rho_v * v
    Xw, Zw = np.meshgrid(g.xc, zc)                     # wall faces: (nz, nx)
    jet = jet_blend(cfg, Xw, Zw) if jet_on else np.zeros((nz, nx))
    T_jet = T_j if jet_on else cfg["T_wall"]
    ref["rhow"] = np.zeros((nz, ny, nx))
    U_ref = pack(ns, nx, ny, nz, ref)
    Xc, Yc = np.meshgrid(g.xc, g.yc)
    Xu, Yu = np.meshgrid(g.xf, g.yc)
    Xv, Yv = np.meshgrid(g.xc, g.yf)
    sig = dict(c=F.sponge(cfg, g, Xc, Yc), xf=F.sponge(cfg, g, Xu, Yu), yf=F.sponge(cfg, g, Xv, Yv))
    sigma = {"c": np.broadcast_to(sig["c"], (nz, ny, nx)),
             "xf": np.broadcast_to(sig["xf"], (nz, ny, nx + 1)),
             "yf": np.broadcast_to(sig["yf"], (nz, ny + 1, nx)),
             "zf": np.broadcast_to(sig["c"], (nz, ny, nx))}
    U0 = U_ref.copy()
    if noise is not None and cfg["noise_amp"] > 0:
        U0 = U_ref * (1.0 + cfg["noise_amp"] * noise)
        f = unpack(ns, nx, ny, nz, U0)
        r = unpack(ns, nx, ny, nz, U_ref)
        f["rhou"][:, :, 0] = r["rhou"][:, :, 0]
        f["rhou"][:, :, nx] = r["rhou"][:, :, nx]
        f["rhov"][:, 0, :] = r["rhov"][:, 0, :]
        f["rhov"][:, ny, :] = r["rhov"][:, ny, :]
    Tw = cfg["T_wall"] + (T_jet - cfg["T_wall"]) * jet
    return Case3D(cfg=cfg, tab=tab, kind=kind, sc=sc, grid=g, nz=nz, zeta=1.0 / dz, zc=zc, zf=zf,
                  U_ref=U_ref, sigma=sigma, U0=U0, jet=jet, T_wall_face=Tw)


def delta4_p(f, axis):
    """Fourth index difference (1, -4, 6, -4, 1) along a periodic axis."""
    return (np.roll(f, 2, axis) - 4.0 * np.roll(f, 1, axis) + 6.0 * f - 4.0 * np.roll(f, -1, axis)
            + np.roll(f, -2, axis))


def gauss9_p(f, axis):
    """The nine-point truncated Gaussian filter along a periodic axis."""
    acc = F.GAUSS9[0] * f
    for d in range(1, 5):
        acc = acc + F.GAUSS9[d] * (np.roll(f, d, axis) + np.roll(f, -d, axis))
    return acc


def filter3(f):
    """x, then y (clamped ends, as in two dimensions), then z (periodic)."""
    return gauss9_p(F.gauss9(F.gauss9(f, 2), 1), 0)


class _Closure:
    """The attributes oracle.flow.closure_nd reads."""

    def __init__(self, case):
        self.sc, self.tab, self.kind, self.cfg = case.sc, case.tab, case.kind, case.cfg


def rhs(case: Case3D, U, return_parts=False):
    cfg, sc, g, tab = case.cfg, case.sc, case.grid, case.tab
    ns, nx, ny, nz = tab.ns, g.nx, g.ny, case.nz
    q = unpack(ns, nx, ny, nz, np.asarray(U, dtype=np.float64))
    Re, Pr = sc.Re, sc.Pr
    wall = bool(cfg["wall"])
    xi_c, xi_f = g.xi_c[None, None, :], g.xi_f[None, None, :]
    eta_c, eta_f = g.eta_c[None, :, None], g.eta_f[None, :, None]
    ze = case.zeta
    rho = q["rho"]
    rhou, rhov, rhow, rhoE = q["rhou"], q["rhov"], q["rhow"], q["rhoE"]
    X_, Y_, Z_ = 2, 1, 0                                       # axes

    # (A) primitives at centres and the closure
    ru_c = C.ifc(rhou, X_)
    rv_c = C.ifc(rhov, Y_)
    rw_c = C.ifc_p(rhow, Z_)
    rho_s = [rho - sum(q[f"rs{s}"] for s in range(1, ns))] + [q[f"rs{s}"] for s in range(1, ns)]
    Y = np.stack([r / rho for r in rho_s])
    u_c, v_c, w_c = ru_c / rho, rv_c / rho, rw_c / rho
    e = rhoE / rho - 0.5 * (u_c * u_c + v_c * v_c + w_c * w_c)
    th = F.closure_nd(_Closure(case), rho, e, Y)
    T, p = th["T"], th["p"]
    H = (rhoE + p) / rho

    # (B) face velocities
    rho_xf = C.icf(rho, X_)
    u_xf = rhou / rho_xf
    rho_yf = C.icf(rho, Y_)
    v_yf = rhov / rho_yf
    rho_zf = C.icf_p(rho, Z_)
    w_zf = rhow / rho_zf

    # (C) velocity gradients: normal ones at centres, cross ones on the edges
    dudx = xi_c * C.dfc(u_xf, X_)
    dvdy = eta_c * C.dfc(v_yf, Y_)
    dwdz = ze * C.dfc_p(w_zf, Z_)
    div = dudx + dvdy + dwdz
    w0 = 0.0 if wall else None
    dudy_xy = eta_f * C.dcf(u_xf, Y_, w0)
    dvdx_xy = xi_f * C.dcf(v_yf, X_)
    u_xy = C.icf(u_xf, Y_, w0)
    v_xy = C.icf(v_yf, X_)
    dudz_xz = ze * C.dcf_p(u_xf, Z_)
    dwdx_xz = xi_f * C.dcf(w_zf, X_)
    u_xz = C.icf_p(u_xf, Z_)
    w_xz = C.icf(w_zf, X_)
    dvdz_yz = ze * C.dcf_p(v_yf, Z_)
    dwdy_yz = eta_f * C.dcf(w_zf, Y_, w0)
    v_yz = C.icf_p(v_yf, Z_)
    w_yz = C.icf(w_zf, Y_, w0)

    # (D) artificial diffusivities at centres
    if cfg["artificial_diffusivity"]:
        dudy_c = C.ifc(C.ifc(dudy_xy, Y_), X_)
        dvdx_c = C.ifc(C.ifc(dvdx_xy, Y_), X_)
        dudz_c = C.ifc_p(C.ifc(dudz_xz, X_), Z_)
        dwdx_c = C.ifc_p(C.ifc(dwdx_xz, X_), Z_)
        dvdz_c = C.ifc_p(C.ifc(dvdz_yz, Y_), Z_)
        dwdy_c = C.ifc_p(C.ifc(dwdy_yz, Y_), Z_)
        S = np.sqrt(dudx * dudx + dvdy * dvdy + dwdz * dwdz + 0.5 * (dudy_c + dvdx_c) ** 2
                    + 0.5 * (dudz_c + dwdx_c) ** 2 + 0.5 * (dvdz_c + dwdy_c) ** 2)
        om2 = (dvdx_c - dudy_c) ** 2 + (dudz_c - dwdx_c) ** 2 + (dwdy_c - dvdz_c) ** 2
        fsw = np.where(div < 0.0, div * div / (div * div + om2 + F.DUCROS_EPS), 0.0)
        dx, dy, dzl = 1.0 / xi_c, 1.0 / eta_c, 1.0 / ze

        def d4(f, l):
            return (F.delta4(f, X_) * dx ** l + F.delta4(f, Y_) * dy ** l + delta4_p(f, Z_) * dzl ** l)

        mu_st = filter3(cfg["C_mu"] * rho * np.abs(d4(S, 2)))
        beta_st = filter3(cfg["C_beta"] * rho * fsw * np.abs(d4(div, 2)))
        kap_st = filter3(cfg["C_kappa"] * rho * th["a"] / T * np.abs(d4(e, 1)))
        D_st = np.stack([filter3(cfg["C_D"] * th["a"] * np.abs(d4(Y[s], 1))) for s in range(ns)])
    else:
        mu_st = beta_st = kap_st = np.zeros_like(rho)
        D_st = np.zeros_like(Y)
    if case.kind != F.KIND_CNEQ:
        D_st = np.zeros_like(Y)
    ie = tab.electron()
    if ie is not None:
        D_st[ie] = 0.0

    # (E) transport coefficients
    mu_e = th["mu"] / Re + mu_st
    K = th["k"] / (Re * Pr) + kap_st
    Gd = th["W"] * (th["D"] / Re + D_st)

    # (F) stresses
    tau_xx = mu_e * (2.0 * dudx - 2.0 / 3.0 * div) + beta_st * div
    tau_yy = mu_e * (2.0 * dvdy - 2.0 / 3.0 * div) + beta_st * div
    tau_zz = mu_e * (2.0 * dwdz - 2.0 / 3.0 * div) + beta_st * div
    mu_x = C.icf(mu_e, X_)
    tau_xy = C.icf(mu_x, Y_) * (dudy_xy + dvdx_xy)
    tau_xz = C.icf_p(mu_x, Z_) * (dudz_xz + dwdx_xz)
    tau_yz = C.icf_p(C.icf(mu_e, Y_), Z_) * (dvdz_yz + dwdy_yz)

    def species_flux(Yf, Gf, dXf, m):
        s_ = np.sum(Gf * dXf, axis=0)
        J = -(Gf * dXf - Yf * s_)
        if ie is not None:
            J = F.zero_current(tab, J)
        return J

    # (G) x-fluxes at x-faces
    Yx = np.stack([C.icf(Y[s], X_) for s in range(ns)])
    Gx = np.stack([C.icf(Gd[s], X_) for s in range(ns)])
    hx = np.stack([C.icf(th["h_s"][s], X_) for s in range(ns)])
    dXdx = np.stack([xi_f * C.dcf(th["X"][s], X_) for s in range(ns)])
    Jx = species_flux(Yx, Gx, dXdx, rhou)
    Fsx = [rhou * Yx[s] + Jx[s] for s in range(ns)]
    qx = -C.icf(K, X_) * xi_f * C.dcf(T, X_) + np.sum(hx * Jx, axis=0)
    FEx = rhou * C.icf(H, X_) + qx - (C.icf(tau_xx, X_) * u_xf + C.ifc(tau_xy, Y_) * C.icf(v_c, X_)
                                      + C.ifc_p(tau_xz, Z_) * C.icf(w_c, X_))

    # (H) y-fluxes at y-faces (wall: T_wall (blended to T_j in the orifice), u = w = 0, no
    # diffusion through the wall)
    Tw = (case.T_wall_face / sc.T_ref) if wall else None
    Yy = np.stack([C.icf(Y[s], Y_) for s in range(ns)])
    Gy = np.stack([C.icf(Gd[s], Y_) for s in range(ns)])
    hy = np.stack([C.icf(th["h_s"][s], Y_) for s in range(ns)])
    dXdy = np.stack([eta_f * C.dcf(th["X"][s], Y_) for s in range(ns)])
    Jy = species_flux(Yy, Gy, dXdy, rhov)
    if wall:
        Jy[:, :, 0, :] = 0.0
    Fsy = [rhov * Yy[s] + Jy[s] for s in range(ns)]
    qy = -C.icf(K, Y_) * eta_f * C.dcf(T, Y_, Tw) + np.sum(hy * Jy, axis=0)
    FEy = rhov * C.icf(H, Y_) + qy - (C.ifc(tau_xy, X_) * C.icf(u_c, Y_, w0)
                                      + C.icf(tau_yy, Y_) * v_yf
                                      + C.ifc_p(tau_yz, Z_) * C.icf(w_c, Y_, w0))

    # (H') z-fluxes at z-faces
    Yz = np.stack([C.icf_p(Y[s], Z_) for s in range(ns)])
    Gz = np.stack([C.icf_p(Gd[s], Z_) for s in range(ns)])
    hz = np.stack([C.icf_p(th["h_s"][s], Z_) for s in range(ns)])
    dXdz = np.stack([ze * C.dcf_p(th["X"][s], Z_) for s in range(ns)])
    Jz = species_flux(Yz, Gz, dXdz, rhow)
    Fsz = [rhow * Yz[s] + Jz[s] for s in range(ns)]
    qz = -C.icf_p(K, Z_) * ze * C.dcf_p(T, Z_) + np.sum(hz * Jz, axis=0)
    FEz = rhow * C.icf_p(H, Z_) + qz - (C.ifc(tau_xz, X_) * C.icf_p(u_c, Z_)
                                        + C.ifc(tau_yz, Y_) * C.icf_p(v_c, Z_)
                                        + C.icf_p(tau_zz, Z_) * w_zf)

    # (I) momentum fluxes: normal ones formed on the faces, interpolated to the centres
    Gxx = C.ifc(rhou * u_xf, X_) + p - tau_xx
    Gyy = C.ifc(rhov * v_yf, Y_) + p - tau_yy
    Gzz = C.ifc_p(rhow * w_zf, Z_) + p - tau_zz
    Gxy = C.icf(rho_xf, Y_) * u_xy * v_xy - tau_xy
    Gxz = C.icf_p(rho_xf, Z_) * u_xz * w_xz - tau_xz
    Gyz = C.icf_p(rho_yf, Z_) * v_yz * w_yz - tau_yz

    # (J) divergences, sources, sponge, boundary rows
    R = {}
    R["rho"] = -(xi_c * C.dfc(rhou, X_) + eta_c * C.dfc(rhov, Y_) + ze * C.dfc_p(rhow, Z_))
    for s in range(1, ns):
        R[f"rs{s}"] = -(xi_c * C.dfc(Fsx[s], X_) + eta_c * C.dfc(Fsy[s], Y_)
                        + ze * C.dfc_p(Fsz[s], Z_)) + th["wdot"][s]
    R["rhoE"] = -(xi_c * C.dfc(FEx, X_) + eta_c * C.dfc(FEy, Y_) + ze * C.dfc_p(FEz, Z_))
    R["rhou"] = -(xi_f * C.dcf(Gxx, X_) + eta_c * C.dfc(Gxy, Y_) + ze * C.dfc_p(Gxz, Z_))
    R["rhov"] = -(xi_c * C.dfc(Gxy, X_) + eta_f * C.dcf(Gyy, Y_) + ze * C.dfc_p(Gyz, Z_))
    R["rhow"] = -(xi_c * C.dfc(Gxz, X_) + eta_c * C.dfc(Gyz, Y_) + ze * C.dcf_p(Gzz, Z_))
    ref = unpack(ns, nx, ny, nz, case.U_ref)
    for name, _ in state_layout(ns, nx, ny, nz):
        sig = case.sigma["xf" if name == "rhou" else "yf" if name == "rhov" else
                         "zf" if name == "rhow" else "c"]
        R[name] = R[name] - sig * (q[name] - ref[name])
    R["rhou"][:, :, 0] = 0.0
    R["rhou"][:, :, nx] = 0.0
    R["rhov"][:, 0, :] = 0.0
    R["rhov"][:, ny, :] = 0.0
    out = pack(ns, nx, ny, nz, R)
    if return_parts:
        xm, ym = g.xi_f.max(), g.eta_f.max()
        fl = {"rho": (rhou, rhov, rhow), "rhoE": (FEx, FEy, FEz), "rhou": (Gxx, Gxy, Gxz),
              "rhov": (Gxy, Gyy, Gyz), "rhow": (Gxz, Gyz, Gzz)}
        for s in range(1, ns):
            fl[f"rs{s}"] = (Fsx[s], Fsy[s], Fsz[s])
        gross = {k: max(np.abs(a).max() * xm, np.abs(b).max() * ym, np.abs(c).max() * ze)
                 for k, (a, b, c) in fl.items()}
        return out, dict(T=T, p=p, th=th, gross=gross, E=rhoE / rho, e=e,
                         ke=0.5 * (u_c * u_c + v_c * v_c + w_c * w_c))
    return out


def parity_tolerance(case: Case3D, U):
    """Per-field absolute tolerance, as oracle.flow.parity_tolerance: 1e-12 max|R_f| + the FP64
    rounding floor of the flux divergence + the sponge term + the temperature conditioning of
    the Arrhenius sources and of the pressure in the momentum and energy fluxes."""
    R, parts = rhs(case, U, return_parts=True)
    g = case.grid
    ns = case.tab.ns
    f = unpack(ns, g.nx, g.ny, case.nz, R)
    tol = {k: F.PARITY_RTOL * np.abs(v).max() + F.PARITY_FLOOR * parts["gross"][k]
           for k, v in f.items()}
    q = unpack(ns, g.nx, g.ny, case.nz, np.asarray(U, dtype=np.float64))
    sig_max = max(float(np.max(v)) for v in case.sigma.values())
    for k in tol:
        tol[k] += 16.0 * 2.0 ** -53 * sig_max * np.abs(q[k]).max()
    T_si = parts["T"] * case.sc.T_ref
    scale = np.abs(parts["E"]) + np.abs(parts["e"]) + parts["ke"]
    if case.kind == F.KIND_CPG:
        dT_rel = 8.0 * 2.0 ** -53 * scale / np.abs(parts["e"])
    else:
        dT_rel = 8.0 * 2.0 ** -53 * scale * case.sc.a ** 2 / (parts["th"]["cv"] * T_si)
    if case.kind == F.KIND_CNEQ and case.tab.reactions:
        ta_max = max(r.Ta for r in case.tab.reactions)
        for s in range(1, ns):
            tol[f"rs{s}"] += np.max(np.abs(parts["th"]["wdot"][s]) * ta_max / T_si * dT_rel)
    # The same temperature conditioning moves the pressure by dp = p dT/T at fixed density; the
    # momentum fluxes carry p and the energy fluxes p times the velocity, and their derivatives
    # multiply that by ||D|| <= 6 and the metric (dT/T already bounds the difference of two
    # evaluations; in three dimensions the spanwise derivative of the pressure, with its uniform
    # metric, has no larger flux term to hide it in).
    # Each derivative sees the pressure error within a few points of where it is evaluated:
    # the largest dp within +-3 points along the derivative's direction, times the local metric.
    from scipy.ndimage import maximum_filter1d
    dp = np.abs(parts["p"]) * dT_rel
    spd = np.sqrt(2.0 * parts["ke"])
    met = (g.xi_c[None, None, :], g.eta_c[None, :, None], case.zeta)
    near = [maximum_filter1d(dp, 7, axis=a, mode="wrap" if a == 0 else "nearest") * m
            for a, m in ((2, met[0]), (1, met[1]), (0, met[2]))]
    near_e = [maximum_filter1d(dp * spd, 7, axis=a, mode="wrap" if a == 0 else "nearest") * m
              for a, m in ((2, met[0]), (1, met[1]), (0, met[2]))]
    for name, k in (("rhou", 0), ("rhov", 1), ("rhow", 2)):
        tol[name] += 6.0 * float(near[k].max())
    tol["rhoE"] += 6.0 * float(max(a.max() for a in near_e))
    return tol, R


def rk_stage(case: Case3D, U, dQ, stage, dt):
    """Williamson two-register RK3 stage, as oracle.flow.rk_stage."""
    R = rhs(case, U)
    dQ = F.RK_A[stage] * dQ + dt * R
    return U + F.RK_B[stage] * dQ, dQ, R
