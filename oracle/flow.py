"""FP64 oracle: right-hand side and explicit stage update of the reacting Navier-Stokes equations.

TEST INFRASTRUCTURE (see oracle/gas.py header). Not used by the product path.

Discrete model (2D, staggered grid of Fig. 1; arrays indexed [j, i] with x fastest):

* centres  (Ny, Nx):     rho, rho_s for every species but the first (N2, omitted, Sec. 2.1), rho*E
* x-faces  (Ny, Nx+1):   rho*u          y-faces (Ny+1, Nx): rho*v
* corners  (Ny+1, Nx+1): tau_xy and the cross momentum fluxes

The right-hand side follows Eqs. (5)-(6) with the stress of Eq. (9) (Stokes' 2/3 restored), the
heat flux of Eq. (10), the algebraic diffusion of Eq. (18) driven by mole-fraction gradients
(Eq. 16), the sponge of Eq. (26), the nondimensionalisation of Eqs. (7)-(8), (11), and an
artificial shear viscosity, bulk viscosity, conductivity and species diffusivity for shock
capturing (Sec. 3.3). Time integration is the two-register third-order Runge-Kutta scheme
(Sec. 3.1). Every step is written in the order it is listed in ``rhs``; the compact operators come
from oracle/compact.py and the closure from oracle/gas.py.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
from scipy.special import erf

from . import compact as C
from . import gas as G

KIND_CNEQ, KIND_FROZEN, KIND_CPG, KIND_TPG, KIND_LTE = "cneq", "frozen", "cpg", "tpg", "lte"
PERFECT_KINDS = (KIND_CPG, KIND_TPG)      # composition irrelevant, no reactions or diffusion
# Local thermodynamic equilibrium (Sec. 2.2.2): the composition follows from (rho, e) and the
# element content of the freestream air; the species fields of the state are carried as passive
# scalars (no diffusion, no sources) and do not enter the closure.

SUTHERLAND_C1 = 1.458e-6      # kg m^-1 s^-1 K^-1/2 (Eq. 24)
SUTHERLAND_TS = 110.4         # K (Eq. 24)
RECOVERY_FACTOR = 0.85
DUCROS_EPS = 1.0e-32
GAUSS9 = (3565.0 / 10368.0, 3091.0 / 12960.0, 1997.0 / 25920.0, 149.0 / 12960.0, 107.0 / 103680.0)

# Williamson low-storage RK3 (two registers): dQ <- A_k dQ + dt R(Q);  Q <- Q + B_k dQ
RK_A = (0.0, -5.0 / 9.0, -153.0 / 128.0)
RK_B = (1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0)


KEYES_C2 = 2.646e-3           # W m^-1 K^-3/2 (Eq. 25)
KEYES_C3 = 245.4              # K (Eq. 25)
KEYES_C4 = 12.0               # K (Eq. 25)
TPG_THETA = 3055.0            # K (Eq. 23)


def sutherland(T):
    """Eq. (24)."""
    return SUTHERLAND_C1 * T ** 1.5 / (T + SUTHERLAND_TS)


def keyes(T):
    """Thermal conductivity of the thermally perfect gas, Eq. (25)."""
    return KEYES_C2 * np.sqrt(T) / (1.0 + (KEYES_C3 / T) * 10.0 ** (-KEYES_C4 / T))


# Thermally perfect gas (Eq. 23), read as the harmonic-oscillator heat capacity
#     c_p(T) = c_p0 (1 + (gamma - 1)/gamma (Theta/T)^2 e^(Theta/T) / (e^(Theta/T) - 1)^2),
# with c_p0 fixed by c_p(T_inf) = c_p,inf. Its integral from 0 is the enthalpy
#     h(T) = c_p0 (T + (gamma - 1)/gamma Theta / (e^(Theta/T) - 1)),
# and the internal energy is e = h - R T with the freestream gas constant R.
def _tpg_shape(x):
    """x^2 e^x / (e^x - 1)^2, written as x^2 e^-x / (1 - e^-x)^2 (no overflow at large x)."""
    x = np.asarray(x, dtype=np.float64)
    d = -np.expm1(-x)
    return x * x * np.exp(-x) / (d * d)


def tpg_cp0(sc):
    return sc.cp / (1.0 + (sc.gamma - 1.0) / sc.gamma * float(_tpg_shape(TPG_THETA / sc.T)))


def tpg_cp(sc, T):
    """c_p(T) of Eq. (23), J/(kg K)."""
    return tpg_cp0(sc) * (1.0 + (sc.gamma - 1.0) / sc.gamma * _tpg_shape(TPG_THETA / T))


def tpg_energy(sc, T):
    """Internal energy e(T) = h(T) - R T of the thermally perfect gas, J/kg."""
    x = TPG_THETA / np.asarray(T, dtype=np.float64)
    h = tpg_cp0(sc) * (T + (sc.gamma - 1.0) / sc.gamma * TPG_THETA * np.exp(-x) / -np.expm1(-x))
    return h - sc.R * T


def tpg_temperature(sc, e, T0=None, rtol=1e-14, maxit=60):
    """Newton inversion of e(T) for the thermally perfect gas (de/dT = c_p - R > 0)."""
    e = np.asarray(e, dtype=np.float64)
    T = np.full(e.shape, sc.T) if T0 is None else np.array(T0, dtype=np.float64)
    for _ in range(maxit):
        dT = (tpg_energy(sc, T) - e) / (tpg_cp(sc, T) - sc.R)
        T = T - dT
        if np.all(np.abs(dT) <= rtol * T):
            break
    return T


@dataclasses.dataclass
class Scales:
    """Freestream reference values of Eq. (7) and the numbers of Eq. (11)."""
    rho: float
    a: float
    T: float
    p: float
    mu: float
    k: float
    cp: float
    gamma: float
    R: float
    T_ref: float
    L_ref: float
    Re: float
    Pr: float
    mach: float


def freestream_scales(tab, kind, cfg) -> Scales:
    Y = np.array(cfg["Y_inf"], dtype=np.float64)[:, None]
    T = np.array([cfg["T_inf"]])
    R = float(G.mixture_gas_constant(tab, Y)[0])
    cv = float(G.mixture_cv(tab, T, Y)[0])
    cp = cv + R
    gamma = cp / cv
    rho = cfg["p_inf"] / (R * cfg["T_inf"])
    a = math.sqrt(gamma * R * cfg["T_inf"])
    if kind == KIND_CPG:
        mu = float(sutherland(cfg["T_inf"]))
        k = mu * cp / cfg["prandtl_cpg"]
    elif kind == KIND_TPG:
        mu = float(sutherland(cfg["T_inf"]))
        k = float(keyes(cfg["T_inf"]))
    else:
        X = G.mole_fractions(tab, Y)
        mu_s = G.species_viscosity(tab, T)
        k_s = G.species_conductivity(tab, T, mu_s)
        mu = float(G.wilke_mix(tab, X, mu_s, mu_s)[0])
        k = float(G.wilke_mix(tab, X, mu_s, k_s)[0])
    Re = cfg["reynolds"]
    return Scales(rho=rho, a=a, T=cfg["T_inf"], p=cfg["p_inf"], mu=mu, k=k, cp=cp, gamma=gamma,
                  R=R, T_ref=(gamma - 1.0) * cfg["T_inf"], L_ref=Re * mu / (rho * a), Re=Re,
                  Pr=mu * cp / k, mach=cfg["mach"])


# ---------------------------------------------------------------------------------------------
# Grid (tensor product of 1-D maps; Eq. 27 and a tanh wall clustering)
# ---------------------------------------------------------------------------------------------

def y_map(cfg, eta):
    """Physical y of the index coordinate eta in [0, Ny] (faces at integers) and dy/deta."""
    y0, y1, ny = cfg["y0"], cfg["y1"], cfg["ny"]
    s = np.asarray(eta, dtype=np.float64) / ny
    kind, q = cfg["y_stretch"], cfg["y_param"]
    if kind == "uniform":
        y = y0 + (y1 - y0) * s
        dy = np.full_like(s, (y1 - y0))
    elif kind == "tanh":
        y = y0 + (y1 - y0) * (1.0 - np.tanh(q * (1.0 - s)) / np.tanh(q))
        dy = (y1 - y0) * q / np.cosh(q * (1.0 - s)) ** 2 / np.tanh(q)
    elif kind == "cubic":
        y = y0 + (y1 - y0) * ((1.0 - q) * s ** 3 + q * s)
        dy = (y1 - y0) * (3.0 * (1.0 - q) * s ** 2 + q)
    else:
        raise ValueError(kind)
    return y, dy / ny


@dataclasses.dataclass
class Grid:
    nx: int
    ny: int
    xc: np.ndarray
    xf: np.ndarray
    yc: np.ndarray
    yf: np.ndarray
    xi_c: np.ndarray      # d(xi)/dx at x-centres
    xi_f: np.ndarray      # at x-faces
    eta_c: np.ndarray     # d(eta)/dy at y-centres
    eta_f: np.ndarray     # at y-faces


def make_grid(cfg) -> Grid:
    nx, ny = cfg["nx"], cfg["ny"]
    dx = (cfg["x1"] - cfg["x0"]) / nx
    xf = cfg["x0"] + dx * np.arange(nx + 1)
    xc = cfg["x0"] + dx * (np.arange(nx) + 0.5)
    yf, dyf = y_map(cfg, np.arange(ny + 1, dtype=np.float64))
    yc, dyc = y_map(cfg, np.arange(ny, dtype=np.float64) + 0.5)
    return Grid(nx, ny, xc, xf, yc, yf, np.full(nx, 1.0 / dx), np.full(nx + 1, 1.0 / dx),
                1.0 / dyc, 1.0 / dyf)


# ---------------------------------------------------------------------------------------------
# Case set-up: reference solution, sponge, initial state
# ---------------------------------------------------------------------------------------------

@dataclasses.dataclass
class Case:
    cfg: dict
    tab: G.GasTable
    kind: str
    sc: Scales
    grid: Grid
    U_ref: dict
    sigma: dict          # sponge strength at 'c', 'xf', 'yf'
    U0: dict


def oblique_shock(M1, theta, gamma):
    """Weak oblique-shock solution of the theta-beta-M relation and the Rankine-Hugoniot jumps.
    Returns beta, p2/p1, rho2/rho1, T2/T1, M2."""
    def deflection(beta):
        return math.atan(2.0 / math.tan(beta) * (M1 ** 2 * math.sin(beta) ** 2 - 1.0)
                         / (M1 ** 2 * (gamma + math.cos(2.0 * beta)) + 2.0))
    mu = math.asin(1.0 / M1)
    lo = mu + 1e-12
    hi = lo
    step = 1.0e-3
    while deflection(hi + step) > deflection(hi):
        hi += step
    if deflection(hi) < theta:
        raise ValueError("deflection beyond the attached-shock limit")
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if deflection(mid) < theta:
            lo = mid
        else:
            hi = mid
    beta = 0.5 * (lo + hi)
    Mn1 = M1 * math.sin(beta)
    p21 = 1.0 + 2.0 * gamma / (gamma + 1.0) * (Mn1 ** 2 - 1.0)
    r21 = (gamma + 1.0) * Mn1 ** 2 / ((gamma - 1.0) * Mn1 ** 2 + 2.0)
    T21 = p21 / r21
    Mn2 = math.sqrt((1.0 + 0.5 * (gamma - 1.0) * Mn1 ** 2) / (gamma * Mn1 ** 2 - 0.5 * (gamma - 1.0)))
    M2 = Mn2 / math.sin(beta - theta)
    return beta, p21, r21, T21, M2


def _primitive_profile(case_cfg, sc, tab, kind, x, y):
    """Reference primitives (T[K], p[Pa], u, v [nondim], Y) at points (x, y)."""
    cfg = case_cfg
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    shape = np.broadcast(x, y).shape
    x = np.broadcast_to(x, shape)
    y = np.broadcast_to(y, shape)

    def edge_profile(Te, pe, ue, ve, Me):
        if cfg["wall"]:
            delta = cfg["delta_coef"] * np.sqrt(x / (sc.Re * sc.mach))
            f = erf(2.0 * (y - cfg["y0"]) / delta)
            Tr = Te * (1.0 + RECOVERY_FACTOR * 0.5 * (sc.gamma - 1.0) * Me ** 2)
            Tw = cfg["T_wall"]
            T = Tw + (Tr - Tw) * f - (Tr - Te) * f * f
        else:
            f = np.ones(shape)
            T = np.full(shape, Te)
        return T, np.full(shape, pe), ue * f, ve * f, f

    T, p, u, v, f = edge_profile(sc.T, sc.p, sc.mach, 0.0, sc.mach)
    if cfg["flow"] == "sbli":
        theta = math.radians(cfg["shock_deflection_deg"])
        beta, p21, r21, T21, M2 = oblique_shock(sc.mach, theta, sc.gamma)
        V2 = M2 * math.sqrt(T21)
        T2, p2, u2, v2, f2 = edge_profile(sc.T * T21, sc.p * p21, V2 * math.cos(theta),
                                          -V2 * math.sin(theta), M2)
        ys = (cfg["shock_x"] - x) * math.tan(beta)
        H = 0.5 * (1.0 + np.tanh((y - ys) / cfg["shock_width"]))
        T = (1.0 - H) * T + H * T2
        p = (1.0 - H) * p + H * p2
        u = (1.0 - H) * u + H * u2
        v = (1.0 - H) * v + H * v2
    Yinf = np.array(cfg["Y_inf"], dtype=np.float64)
    Y = np.zeros((tab.ns,) + shape)
    seeded = cfg["wall"] and kind in (KIND_CNEQ, KIND_FROZEN)
    m = cfg["minor_species"] * 4.0 * f * (1.0 - f) if seeded else 0.0 * f
    names = [s.name for s in tab.species]
    Y[:] = Yinf.reshape((-1,) + (1,) * len(shape))
    Y[names.index("N2")] = Yinf[names.index("N2")] * (1.0 - m)
    Y[names.index("O2")] = Yinf[names.index("O2")] * (1.0 - m)
    Y[names.index("NO")] = 0.5 * m
    Y[names.index("N")] = 0.2 * m
    Y[names.index("O")] = 0.3 * m
    return T, p, u, v, Y


def _conserved_from_primitive(tab, kind, sc, T, p, u, v, Y):
    """Nondimensional rho, rho_s, rho*E at points given SI T, p and nondim u, v."""
    flatT = T.ravel()
    flatY = Y.reshape(tab.ns, -1)
    if kind == KIND_CPG:
        rho_si = p.ravel() / (sc.R * flatT)
        e_nd = (flatT / sc.T_ref) / sc.gamma
    elif kind == KIND_TPG:
        rho_si = p.ravel() / (sc.R * flatT)
        e_nd = tpg_energy(sc, flatT) / sc.a ** 2
    elif kind == KIND_LTE:
        # density from the profile's T and p with the gas constant of the air, then the
        # equilibrium composition and energy at that (T, rho)
        rho_si = p.ravel() / (G.mixture_gas_constant(tab, flatY) * flatT)
        Yeq, e_si, _, _ = G.equilibrium_at(tab, flatT, rho_si, G.element_content(tab, flatY))
        flatY = Yeq
        e_nd = e_si / sc.a ** 2
        Y = Yeq.reshape(Y.shape)
    else:
        rho_si = p.ravel() / (G.mixture_gas_constant(tab, flatY) * flatT)
        e_nd = G.mixture_energy(tab, flatT, flatY) / sc.a ** 2
    rho = (rho_si / sc.rho).reshape(T.shape)
    e_nd = e_nd.reshape(T.shape)
    rhoE = rho * (e_nd + 0.5 * (u * u + v * v))
    return rho, rho * Y, rhoE


STATE_FIELDS = None   # documented layout: rho, rho_s[1..ns-1], rhoE at centres; rhou; rhov


def state_layout(ns, nx, ny):
    """Offsets of the canonical state vector: (name, shape) in order."""
    out = [("rho", (ny, nx))]
    out += [(f"rs{s}", (ny, nx)) for s in range(1, ns)]
    out += [("rhoE", (ny, nx)), ("rhou", (ny, nx + 1)), ("rhov", (ny + 1, nx))]
    return out


def pack(ns, nx, ny, fields):
    return np.concatenate([np.asarray(fields[name], dtype=np.float64).ravel()
                           for name, _ in state_layout(ns, nx, ny)])


def unpack(ns, nx, ny, U):
    out, off = {}, 0
    for name, shape in state_layout(ns, nx, ny):
        size = shape[0] * shape[1]
        out[name] = np.asarray(U[off:off + size]).reshape(shape)
        off += size
    assert off == U.size
    return out


def sponge(cfg, grid, x, y):
    """sigma(x, y) = sigma_max (r_in^3 + r_out^3 + r_top^3): cubic ramps inside each zone (Eq. 26)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    s = np.zeros(np.broadcast(x, y).shape)
    if cfg["sponge_in"] > 0:
        r = np.clip((cfg["x0"] + cfg["sponge_in"] - x) / cfg["sponge_in"], 0.0, 1.0)
        s = s + r ** 3
    if cfg["sponge_out"] > 0:
        r = np.clip((x - (cfg["x1"] - cfg["sponge_out"])) / cfg["sponge_out"], 0.0, 1.0)
        s = s + r ** 3
    ntop = cfg["sponge_top_cells"]
    if ntop > 0:
        ytop = grid.yf[cfg["ny"] - ntop]
        r = np.clip((y - ytop) / (cfg["y1"] - ytop), 0.0, 1.0)
        s = s + r ** 3
    return cfg["sponge_sigma"] * s


def make_case(cfg, tab, noise=None) -> Case:
    kind = cfg["kind"]
    if kind == KIND_LTE and tab.electron() is not None:
        raise ValueError("the LTE closure conserves N and O only: no charged species")
    if len(cfg["Y_inf"]) != tab.ns:
        raise ValueError("Y_inf must list one mass fraction per species of the table")
    sc = freestream_scales(tab, kind, cfg)
    g = make_grid(cfg)
    nx, ny, ns = g.nx, g.ny, tab.ns
    Xc, Yc = np.meshgrid(g.xc, g.yc)
    Xu, Yu = np.meshgrid(g.xf, g.yc)
    Xv, Yv = np.meshgrid(g.xc, g.yf)
    ref = {}
    T, p, u, v, Y = _primitive_profile(cfg, sc, tab, kind, Xc, Yc)
    rho, rhoY, rhoE = _conserved_from_primitive(tab, kind, sc, T, p, u, v, Y)
    ref["rho"] = rho
    for s in range(1, ns):
        ref[f"rs{s}"] = rhoY[s]
    ref["rhoE"] = rhoE
    T, p, u, v, Y = _primitive_profile(cfg, sc, tab, kind, Xu, Yu)
    rho_u, _, _ = _conserved_from_primitive(tab, kind, sc, T, p, u, v, Y)
    ref["rhou"] = rho_u * u
    T, p, u, v, Y = _primitive_profile(cfg, sc, tab, kind, Xv, Yv)
    rho_v, _, _ = _conserved_from_primitive(tab, kind, sc, T, p, u, v, Y)
    ref["rhov"] = rho_v * v
    T, p, u, v, Y = _primitive_profile(cfg, sc, tab, kind, Xu[:, :1], Yu[:, :1])
    rho_in, rhoY_in, rhoE_in = _conserved_from_primitive(tab, kind, sc, T, p, u, v, Y)
    p_nd = p / (sc.rho * sc.a ** 2)
    inflow = dict(rho=rho_in[:, 0], Y=(rhoY_in / rho_in)[:, :, 0],
                  H=((rhoE_in + p_nd) / rho_in)[:, 0])
    sigma = dict(c=sponge(cfg, g, Xc, Yc), xf=sponge(cfg, g, Xu, Yu), yf=sponge(cfg, g, Xv, Yv))
    U_ref = pack(ns, nx, ny, ref)
    U0 = U_ref.copy()
    if noise is not None and cfg["noise_amp"] > 0:
        U0 = U_ref * (1.0 + cfg["noise_amp"] * noise)
        f = unpack(ns, nx, ny, U0)
        r = unpack(ns, nx, ny, U_ref)
        f["rhou"][:, 0] = r["rhou"][:, 0]
        f["rhou"][:, nx] = r["rhou"][:, nx]
        f["rhov"][0, :] = r["rhov"][0, :]
        f["rhov"][ny, :] = r["rhov"][ny, :]
    case = Case(cfg=cfg, tab=tab, kind=kind, sc=sc, grid=g, U_ref=U_ref, sigma=sigma, U0=U0)
    case.inflow = inflow
    return case


# ---------------------------------------------------------------------------------------------
# Pointwise closure in nondimensional variables
# ---------------------------------------------------------------------------------------------

def closure_nd(case: Case, rho, e, Y):
    """Nondimensional T, p, h_s, w_s, mu, k, D_s, X_s, W_s = rho M_s / M_mix, frozen sound speed."""
    sc, tab, kind = case.sc, case.tab, case.kind
    shape = rho.shape
    r1 = rho.ravel()
    e1 = e.ravel()
    Y1 = Y.reshape(tab.ns, -1)
    ns = tab.ns
    if kind == KIND_CPG:
        T = sc.gamma * e1
        p = r1 * (sc.gamma - 1.0) / sc.gamma * T
        mu = sutherland(T * sc.T_ref) / sc.mu
        out = dict(T=T, p=p, h_s=np.zeros_like(Y1), wdot=np.zeros_like(Y1), mu=mu, k=mu,
                   D=np.zeros_like(Y1), X=np.zeros_like(Y1), W=np.zeros_like(Y1),
                   a=np.sqrt(sc.gamma * p / r1))
    elif kind == KIND_TPG:
        T_si = tpg_temperature(sc, e1 * sc.a ** 2)
        T = T_si / sc.T_ref
        p = r1 * (sc.gamma - 1.0) / sc.gamma * T                  # Eq. (22)
        cp = tpg_cp(sc, T_si)
        gam = cp / (cp - sc.R)
        out = dict(T=T, p=p, h_s=np.zeros_like(Y1), wdot=np.zeros_like(Y1),
                   mu=sutherland(T_si) / sc.mu, k=keyes(T_si) / sc.k,
                   D=np.zeros_like(Y1), X=np.zeros_like(Y1), W=np.zeros_like(Y1),
                   a=np.sqrt(gam * p / r1))
    elif kind == KIND_LTE:
        bm = G.element_content(tab, np.array(case.cfg["Y_inf"], dtype=np.float64))
        th = G.lte_eval(tab, r1 * sc.rho, e1 * sc.a ** 2, bm)
        out = dict(T=th["T"] / sc.T_ref, p=th["p"] / (sc.rho * sc.a ** 2),
                   h_s=np.zeros_like(Y1), wdot=np.zeros_like(Y1), mu=th["mu"] / sc.mu,
                   k=th["k"] / sc.k, D=np.zeros_like(Y1), X=th["X"], W=np.zeros_like(Y1),
                   a=th["a"] / sc.a, cv=th["cv"])
    else:
        th = G.thermo_eval(tab, r1 * sc.rho, e1 * sc.a ** 2, Y1, reactions=(kind == KIND_CNEQ))
        M = tab.M()[:, None]
        Mmix = 1.0 / np.sum(Y1 / M, axis=0)
        diffusive = kind == KIND_CNEQ
        out = dict(T=th["T"] / sc.T_ref, p=th["p"] / (sc.rho * sc.a ** 2),
                   h_s=th["h_s"] / sc.a ** 2,
                   wdot=th["wdot"] * sc.L_ref / (sc.rho * sc.a),
                   mu=th["mu"] / sc.mu, k=th["k"] / sc.k,
                   D=(th["D"] * sc.rho / sc.mu) if diffusive else np.zeros_like(Y1),
                   X=th["X"], W=(r1 * M / Mmix) if diffusive else np.zeros_like(Y1),
                   a=th["a"] / sc.a, cv=th["cv"])
    res = {}
    for key, val in out.items():
        res[key] = val.reshape((ns,) + shape) if val.ndim == 2 else val.reshape(shape)
    return res


# ---------------------------------------------------------------------------------------------
# Stefan-Maxwell diffusion (Eq. 17), the alternative to the algebraic model of Eq. (18)
# ---------------------------------------------------------------------------------------------
# Eq. (17) with the interaction coefficients of the Stefan-Maxwell relations,
#     d_s = sum_{i != s} X_s X_i (V_i - V_s) / D_si,   d_s = grad X_s (Eq. 16),
# written for the fluxes J_s = rho Y_s V_s (X_i / Y_i = Mbar / M_i), which stays regular for
# vanishing mole fractions:
#     sum_{i != s} (X_s J_i / M_i - X_i J_s / M_s) / D_si = (rho / Mbar) d_s,
# with the equation of the first species (the omitted, most abundant one) replaced by the
# mass constraint sum_s J_s = 0. Nondimensional D_si = D_si rho_inf / (mu_inf Re), so J carries
# 1/Re like the algebraic flux. Evaluated at the faces from the interpolated density and mass
# fractions, the face gradients of X and binary coefficients at the interpolated T and p.
DIFF_RAMSHAW, DIFF_SM = "ramshaw", "stefan_maxwell"


def stefan_maxwell_fluxes(tab, rho_f, Y_f, dX_f, Dnd):
    """J_s at face points. rho_f (n,), Y_f and dX_f (ns, n), Dnd (ns, ns, n) nondimensional
    binary coefficients including 1/Re. Returns (ns, n)."""
    ns = tab.ns
    M = tab.M()
    n = rho_f.size
    inv = Y_f / M[:, None]
    Mbar = 1.0 / np.sum(inv, axis=0)
    X = inv * Mbar
    A = np.zeros((n, ns, ns))
    b = np.zeros((n, ns))
    for s in range(1, ns):
        for i in range(ns):
            if i != s:
                A[:, s, i] += X[s] / (M[i] * Dnd[s, i])
                A[:, s, s] -= X[i] / (M[s] * Dnd[s, i])
        b[:, s] = rho_f / Mbar * dX_f[s]
    A[:, 0, :] = 1.0
    return np.linalg.solve(A, b[..., None])[..., 0].T


def _sm_face_fluxes(case, rho_f, Y_f, dX_f, T_f, p_f):
    sc, tab = case.sc, case.tab
    shape = rho_f.shape
    T_si = T_f.ravel() * sc.T_ref
    p_si = p_f.ravel() * sc.rho * sc.a ** 2
    Dnd = G.binary_diffusion(tab, T_si, p_si) * sc.rho / sc.mu / sc.Re
    J = stefan_maxwell_fluxes(tab, rho_f.ravel(), Y_f.reshape(tab.ns, -1),
                              dX_f.reshape(tab.ns, -1), Dnd)
    return J.reshape((tab.ns,) + shape)


# ---------------------------------------------------------------------------------------------
# Artificial diffusivity helpers (Sec. 3.3)
# ---------------------------------------------------------------------------------------------

def zero_current(tab, J):
    """Charged mixtures (reading; the paper treats neutral air only): the electrons diffuse with
    the ions, so the conduction current vanishes, J_e = M_e sum_ions J_i / M_i, and the omitted
    first species takes J_0 = -sum_{s >= 1} J_s so that the diffusive mass fluxes still sum to
    zero. J: (ns, ...) fluxes of Eq. (18) with ambipolar ion coefficients."""
    ie = tab.electron()
    M = tab.M()
    J = np.array(J, dtype=np.float64, copy=True)
    acc = np.zeros_like(J[0])
    for i in range(tab.ns):
        if tab.species[i].charge > 0:
            acc = acc + J[i] / M[i]
    J[ie] = M[ie] * acc
    tot = np.zeros_like(J[0])
    for i in range(1, tab.ns):
        tot = tot + J[i]
    J[0] = -tot
    return J


def delta4(f, axis):
    """Fourth index difference (1, -4, 6, -4, 1); the two rows nearest each end reuse the
    stencil centred on the nearest row where it fits."""
    fm = np.moveaxis(f, axis, 0)
    n = fm.shape[0]
    out = np.empty_like(fm)
    for i in range(n):
        c = min(max(i, 2), n - 3)
        out[i] = fm[c - 2] - 4.0 * fm[c - 1] + 6.0 * fm[c] - 4.0 * fm[c + 1] + fm[c + 2]
    return np.moveaxis(out, 0, axis)


def gauss9(f, axis):
    """Nine-point truncated Gaussian filter; indices beyond the ends take the end value."""
    fm = np.moveaxis(f, axis, 0)
    n = fm.shape[0]
    out = np.zeros_like(fm)
    for i in range(n):
        acc = GAUSS9[0] * fm[i]
        for d in range(1, 5):
            acc = acc + GAUSS9[d] * (fm[max(i - d, 0)] + fm[min(i + d, n - 1)])
        out[i] = acc
    return np.moveaxis(out, 0, axis)


def filter2(f):
    """The Gaussian filter along x (axis 1), then along y (axis 0)."""
    return gauss9(gauss9(f, 1), 0)


def ducros(div, omega):
    """Ducros switch H(-div u) (div u)^2 / ((div u)^2 + |omega|^2 + eps)."""
    return np.where(div < 0.0, div * div / (div * div + omega * omega + DUCROS_EPS), 0.0)


def artificial_diffusivity(cfg, rho, a, T, e, Y, dudx, dvdy, dudy_c, dvdx_c, dx, dy):
    """Artificial shear viscosity, bulk viscosity, conductivity and species diffusivities at the
    centres (Sec. 3.3, in the form of the localized-artificial-diffusivity papers it cites):
        mu*  = C_mu    rho           |sum_l d4_l(S) dl^2|~
        beta* = C_beta rho f_sw      |sum_l d4_l(div u) dl^2|~
        kappa* = C_kappa rho a / T   |sum_l d4_l(e) dl|~
        D*_s = C_D a                 |sum_l d4_l(Y_s) dl|~
    with S = (dudx^2 + dvdy^2 + (dudy + dvdx)^2 / 2)^(1/2), omega = dvdx - dudy, d4_l the fourth
    index difference along direction l (delta4), dl the local cell size (dx varies along axis 1,
    dy along axis 0) and ~ the Gaussian filter in x then y (filter2). Arrays are (ny, nx) at the
    centres; Y is (ns, ny, nx). Returns (mu*, beta*, kappa*, D*)."""
    S = np.sqrt(dudx * dudx + dvdy * dvdy + 0.5 * (dudy_c + dvdx_c) ** 2)
    div = dudx + dvdy
    fsw = ducros(div, dvdx_c - dudy_c)
    mu_st = filter2(cfg["C_mu"] * rho * np.abs(delta4(S, 1) * dx * dx + delta4(S, 0) * dy * dy))
    beta_st = filter2(cfg["C_beta"] * rho * fsw
                      * np.abs(delta4(div, 1) * dx * dx + delta4(div, 0) * dy * dy))
    kap_st = filter2(cfg["C_kappa"] * rho * a / T
                     * np.abs(delta4(e, 1) * dx + delta4(e, 0) * dy))
    D_st = np.stack([filter2(cfg["C_D"] * a
                             * np.abs(delta4(Y[s], 1) * dx + delta4(Y[s], 0) * dy))
                     for s in range(Y.shape[0])])
    return mu_st, beta_st, kap_st, D_st


# ---------------------------------------------------------------------------------------------
# The right-hand side
# ---------------------------------------------------------------------------------------------

def rhs(case: Case, U, return_parts=False):
    cfg, sc, g, tab = case.cfg, case.sc, case.grid, case.tab
    ns, nx, ny = tab.ns, g.nx, g.ny
    q = unpack(ns, nx, ny, np.asarray(U, dtype=np.float64))
    Re, Pr = sc.Re, sc.Pr
    wall = bool(cfg["wall"])
    xi_c = g.xi_c[None, :]
    xi_f = g.xi_f[None, :]
    eta_c = g.eta_c[:, None]
    eta_f = g.eta_f[:, None]
    rho = q["rho"]
    rhou, rhov, rhoE = q["rhou"], q["rhov"], q["rhoE"]

    # (A) primitives at centres (face momenta interpolated to centres; omitted species recovered)
    ru_c = C.ifc(rhou, 1)
    rv_c = C.ifc(rhov, 0)
    rho_s = [rho - sum(q[f"rs{s}"] for s in range(1, ns))] + [q[f"rs{s}"] for s in range(1, ns)]
    Y = np.stack([r / rho for r in rho_s])
    u_c = ru_c / rho
    v_c = rv_c / rho
    e = rhoE / rho - 0.5 * (u_c * u_c + v_c * v_c)          # Eq. (8) with Ec = 1
    th = closure_nd(case, rho, e, Y)
    T, p = th["T"], th["p"]
    H = (rhoE + p) / rho

    # (B) face velocities
    inf = case.inflow if cfg.get("_inflow_dirichlet") else None
    rho_xf = C.icf(rho, 1, None if inf is None else inf["rho"])
    u_xf = rhou / rho_xf
    rho_yf = C.icf(rho, 0)
    v_yf = rhov / rho_yf

    # (C) velocity gradients: normal ones at centres, cross ones at corners
    dudx = xi_c * C.dfc(u_xf, 1)
    dvdy = eta_c * C.dfc(v_yf, 0)
    div = dudx + dvdy
    uwall = 0.0 if wall else None
    dudy_cn = eta_f * C.dcf(u_xf, 0, uwall)
    dvdx_cn = xi_f * C.dcf(v_yf, 1)
    u_cn = C.icf(u_xf, 0, uwall)
    v_cn = C.icf(v_yf, 1)

    # (D) artificial diffusivities at centres
    if cfg["artificial_diffusivity"]:
        dudy_c = C.ifc(C.ifc(dudy_cn, 0), 1)
        dvdx_c = C.ifc(C.ifc(dvdx_cn, 0), 1)
        mu_st, beta_st, kap_st, D_st = artificial_diffusivity(
            cfg, rho, th["a"], T, e, Y, dudx, dvdy, dudy_c, dvdx_c, 1.0 / xi_c, 1.0 / eta_c)
    else:
        mu_st = beta_st = kap_st = np.zeros_like(rho)
        D_st = np.zeros_like(Y)
    if case.kind != KIND_CNEQ:
        D_st = np.zeros_like(Y)
    ie = tab.electron()
    if ie is not None:
        D_st[ie] = 0.0          # the electron flux follows the ions (zero_current)

    # (E) transport coefficients (viscous scale 1/Re, conduction 1/(Re Pr Ec), diffusion 1/Re)
    mu_e = th["mu"] / Re + mu_st
    K = th["k"] / (Re * Pr) + kap_st
    sm = case.kind == KIND_CNEQ and cfg.get("diffusion_model", DIFF_RAMSHAW) == DIFF_SM
    if sm and ie is not None:
        raise ValueError("Stefan-Maxwell diffusion is not defined here for charged mixtures")
    # with Stefan-Maxwell diffusion the algebraic form keeps only the artificial diffusivity
    Gd = th["W"] * ((0.0 if sm else th["D"] / Re) + D_st)

    # (F) viscous stresses, Eq. (9) with the Stokes 2/3 and the artificial bulk viscosity
    tau_xx = mu_e * (2.0 * dudx - 2.0 / 3.0 * div) + beta_st * div
    tau_yy = mu_e * (2.0 * dvdy - 2.0 / 3.0 * div) + beta_st * div
    mu_cn = C.icf(C.icf(mu_e, 1), 0)
    tau_xy = mu_cn * (dudy_cn + dvdx_cn)

    # (G) x-fluxes at x-faces
    Yx = np.stack([C.icf(Y[s], 1, None if inf is None else inf["Y"][s]) for s in range(ns)])
    Gx = np.stack([C.icf(Gd[s], 1) for s in range(ns)])
    hx = np.stack([C.icf(th["h_s"][s], 1) for s in range(ns)])
    dXdx = np.stack([xi_f * C.dcf(th["X"][s], 1) for s in range(ns)])
    Hx = C.icf(H, 1, None if inf is None else inf["H"])
    Kx = C.icf(K, 1)
    dTdx = xi_f * C.dcf(T, 1)
    txx_x = C.icf(tau_xx, 1)
    v_x = C.icf(v_c, 1)
    txy_x = C.ifc(tau_xy, 0)
    sumx = np.sum(Gx * dXdx, axis=0)
    Jx = -(Gx * dXdx - Yx * sumx)                            # Eq. (18), gradient of X (Eq. 16)
    if sm:
        Jx = Jx + _sm_face_fluxes(case, rho_xf, Yx, dXdx, C.icf(T, 1), C.icf(p, 1))
    if ie is not None:
        Jx = zero_current(tab, Jx)
    Fsx = [rhou * Yx[s] + Jx[s] for s in range(ns)]
    qx = -Kx * dTdx + np.sum(hx * Jx, axis=0)                # Eq. (10)
    FEx = rhou * Hx + qx - (txx_x * u_xf + txy_x * v_x)

    # (H) y-fluxes at y-faces (wall: T = T_w, u = 0, no diffusion through the wall)
    Tw = cfg["T_wall"] / sc.T_ref if wall else None
    Yy = np.stack([C.icf(Y[s], 0) for s in range(ns)])
    Gy = np.stack([C.icf(Gd[s], 0) for s in range(ns)])
    hy = np.stack([C.icf(th["h_s"][s], 0) for s in range(ns)])
    dXdy = np.stack([eta_f * C.dcf(th["X"][s], 0) for s in range(ns)])
    Hy = C.icf(H, 0)
    Ky = C.icf(K, 0)
    dTdy = eta_f * C.dcf(T, 0, Tw)
    tyy_y = C.icf(tau_yy, 0)
    u_y = C.icf(u_c, 0, uwall)
    txy_y = C.ifc(tau_xy, 1)
    sumy = np.sum(Gy * dXdy, axis=0)
    Jy = -(Gy * dXdy - Yy * sumy)
    if sm:
        Jy = Jy + _sm_face_fluxes(case, rho_yf, Yy, dXdy, C.icf(T, 0), C.icf(p, 0))
    if ie is not None:
        Jy = zero_current(tab, Jy)
    if wall:
        Jy[:, 0, :] = 0.0
    Fsy = [rhov * Yy[s] + Jy[s] for s in range(ns)]
    qy = -Ky * dTdy + np.sum(hy * Jy, axis=0)
    FEy = rhov * Hy + qy - (txy_y * u_y + tyy_y * v_yf)

    # (I) momentum fluxes. The normal flux rho u u is formed on the faces from the face momentum
    # and the face velocity, then interpolated to the centres: with the centre product
    # (I_fc m)^2 / rho the linearised scheme is unstable for supersonic flow even on a periodic
    # grid, because I_cf I_fc differs from 1 at grid scale while the energy flux sees m directly.
    Gxx = C.ifc(rhou * u_xf, 1) + p - tau_xx
    Gyy = C.ifc(rhov * v_yf, 0) + p - tau_yy
    rho_cn = C.icf(rho_xf, 0)
    Gxy = rho_cn * u_cn * v_cn - tau_xy

    # (J) divergences, sources, sponge, boundary rows
    R = {}
    R["rho"] = -(xi_c * C.dfc(rhou, 1) + eta_c * C.dfc(rhov, 0))
    for s in range(1, ns):
        R[f"rs{s}"] = -(xi_c * C.dfc(Fsx[s], 1) + eta_c * C.dfc(Fsy[s], 0)) + th["wdot"][s]
    R["rhoE"] = -(xi_c * C.dfc(FEx, 1) + eta_c * C.dfc(FEy, 0))
    R["rhou"] = -(xi_f * C.dcf(Gxx, 1) + eta_c * C.dfc(Gxy, 0))
    R["rhov"] = -(xi_c * C.dfc(Gxy, 1) + eta_f * C.dcf(Gyy, 0))
    ref = unpack(ns, nx, ny, case.U_ref)
    for name, _ in state_layout(ns, nx, ny):
        sig = case.sigma["xf" if name == "rhou" else "yf" if name == "rhov" else "c"]
        R[name] = R[name] - sig * (q[name] - ref[name])
    R["rhou"][:, 0] = 0.0
    for c in range(cfg.get("_fix_cols", 0)):
        for name in R:
            if name == "rhou":
                R[name][:, c + 1] = 0.0
            else:
                R[name][:, c] = 0.0
    if not cfg.get("_free_outflow"):
        R["rhou"][:, nx] = 0.0
    if wall or not cfg.get("_free_bottom"):
        R["rhov"][0, :] = 0.0
    if not cfg.get("_free_top"):
        R["rhov"][ny, :] = 0.0
    out = pack(ns, nx, ny, R)
    if return_parts:
        # largest |flux| x |metric| entering each field's divergence (for rounding-floor bounds)
        xm, ym = g.xi_f.max(), g.eta_f.max()
        gross = {"rho": max(np.abs(rhou).max() * xm, np.abs(rhov).max() * ym),
                 "rhoE": max(np.abs(FEx).max() * xm, np.abs(FEy).max() * ym),
                 "rhou": max(np.abs(Gxx).max() * xm, np.abs(Gxy).max() * ym),
                 "rhov": max(np.abs(Gxy).max() * xm, np.abs(Gyy).max() * ym)}
        for s in range(1, ns):
            gross[f"rs{s}"] = max(np.abs(Fsx[s]).max() * xm, np.abs(Fsy[s]).max() * ym)
        return out, dict(T=T, p=p, th=th, mu_st=mu_st, beta_st=beta_st, kap_st=kap_st, D_st=D_st,
                         tau_xy=tau_xy, dTdy=dTdy, gross=gross, E=rhoE / rho, e=e,
                         ke=0.5 * (u_c * u_c + v_c * v_c))
    return out


# Parity criterion for a computed right-hand side against this oracle (test infrastructure).
# One FP64 evaluation of -metric * D(F) is off by up to about 8 eps ||D||_inf max|F| max|metric|,
# so two that round in different orders differ by up to twice that; ||D||_inf <= 6 bounds the compact derivative with its
# closures (row sums of |B| <= 4.3, ||A^-1||_inf <= 1/(1 - 2 alpha) = 1.41). The stated
# 1e-12 normwise tolerance applies on top of that floor.
PARITY_RTOL = 1.0e-12
PARITY_FLOOR = 16.0 * 2.0 ** -53 * 6.0


# The species sources w_s carry exp(-T_a/T): a relative temperature difference dT/T between two
# converged inversions changes them by (T_a/T) dT/T. Two FP64 evaluations of e = E - |u|^2/2 and
# of the Newton residual differ by a few eps (|E| + |e| + |u|^2/2) a_inf^2, which moves T by that
# over c_v; the tolerance adds max_i |w_s,i| (T_a,max / T_i) (dT/T)_i with that estimate (times 8).
def parity_tolerance(case: Case, U):
    """Per-field absolute tolerance: 1e-12 max|R_f| + 8 eps ||D|| max|F_f| max|metric|, plus the
    sponge term, the temperature conditioning of the Arrhenius sources and of the pressure in the
    momentum and energy fluxes."""
    R, parts = rhs(case, U, return_parts=True)
    g = case.grid
    f = unpack(case.tab.ns, g.nx, g.ny, R)
    tol = {k: PARITY_RTOL * np.abs(v).max() + PARITY_FLOOR * parts["gross"][k]
           for k, v in f.items()}
    # sponge term sigma (U - U_ref): U and U_ref agree to the seeded noise, so the difference
    # carries the rounding of U itself (a few eps |U|) times sigma
    q = unpack(case.tab.ns, g.nx, g.ny, np.asarray(U, dtype=np.float64))
    sig_max = max(float(np.max(v)) for v in case.sigma.values())
    for k in tol:
        tol[k] += 16.0 * 2.0 ** -53 * sig_max * np.abs(q[k]).max()
    T_si = parts["T"] * case.sc.T_ref
    scale = np.abs(parts["E"]) + np.abs(parts["e"]) + parts["ke"]
    if case.kind == KIND_CPG:
        dT_rel = 8.0 * 2.0 ** -53 * scale / np.abs(parts["e"])
    elif case.kind == KIND_TPG:
        cv = tpg_cp(case.sc, T_si) - case.sc.R
        dT_rel = 8.0 * 2.0 ** -53 * scale * case.sc.a ** 2 / (cv * T_si)
    else:
        dT_rel = 8.0 * 2.0 ** -53 * scale * case.sc.a ** 2 / (parts["th"]["cv"] * T_si)
    if case.kind == KIND_CNEQ and case.tab.reactions:
        ta_max = max(r.Ta for r in case.tab.reactions)
        for s in range(1, case.tab.ns):
            tol[f"rs{s}"] += np.max(np.abs(parts["th"]["wdot"][s]) * ta_max / T_si * dT_rel)
    # The same temperature conditioning moves the pressure by dp = p dT/T at fixed density
    # (Eq. 8 for the perfect gases, p = rho R T of the mixture otherwise); the momentum fluxes
    # carry p and the energy fluxes p times the velocity, and their derivatives multiply that by
    # ||D|| <= 6 and the metric (dT/T above already bounds the difference of two evaluations).
    # Each derivative sees the pressure within a few points of where it is evaluated: the largest
    # dp within +-3 points along its direction, times the local metric.
    from scipy.ndimage import maximum_filter1d
    dp = np.abs(parts["p"]) * dT_rel
    spd = np.sqrt(2.0 * parts["ke"])
    mets = ((1, g.xi_c[None, :]), (0, g.eta_c[:, None]))
    near = [maximum_filter1d(dp, 7, axis=a, mode="nearest") * m for a, m in mets]
    near_e = [maximum_filter1d(dp * spd, 7, axis=a, mode="nearest") * m for a, m in mets]
    tol["rhou"] += 6.0 * float(near[0].max())
    tol["rhov"] += 6.0 * float(near[1].max())
    tol["rhoE"] += 6.0 * float(max(a.max() for a in near_e))
    if case.kind == KIND_LTE:
        # The reference partial densities of an LTE case are an equilibrium composition,
        # c_s = (p_std / (R T)) exp(a_s . lambda - G_s / (R T)). Two correct evaluations round
        # that exponent differently by a few eps times its size (|G_s / (R T)| reaches ~200 for
        # the atoms near 300 K), which moves each c_s relatively by as much; the sponge term
        # sigma (Q - Q_ref) carries it into the passive species fields.
        T_si = parts["T"] * case.sc.T_ref
        g_max = max(float(np.max(np.abs(G.species_gibbs_over_rt(sp, np.array([T_si.min(), T_si.max()])))))
                    for sp in case.tab.species)
        ref = unpack(case.tab.ns, g.nx, g.ny, case.U_ref)
        for s in range(1, case.tab.ns):
            tol[f"rs{s}"] += sig_max * 8.0 * 2.0 ** -53 * g_max * np.abs(ref[f"rs{s}"]).max()
    return tol, R


# ---------------------------------------------------------------------------------------------
# Low-pass filter of the conserved state (after each RK step when the case sets filter_sigma)
# ---------------------------------------------------------------------------------------------
# The shock capturing of Sec. 3.3 follows the localized-artificial-diffusivity papers it cites,
# which run their non-dissipative compact schemes together with a high-order low-pass filter of
# the conserved variables; the paper does not spell one out. Reading: along every grid line of
# every field, f_i <- f_i - sigma (D_m f)_i with the 2m-th order difference
#     (D_m f)_i = 4^-m sum_{n=-m..m} (-1)^n C(2m, m+n) f_{i+n},
# whose Fourier symbol is sin^(2m)(theta/2) (1 at the grid-to-grid mode, O(theta^(2m)) for smooth
# data). m = 5 where the stencil fits; at distance d < 5 from either end of the line m = d, and
# the end points themselves are left unchanged. The x pass runs first, the y pass on its result.
FILTER_ORDER_HALF = 5


def filter_weights(m):
    """Weights of (D_m f)_i on f_{i-m} .. f_{i+m}."""
    return np.array([(-1) ** n * math.comb(2 * m, m + n) for n in range(-m, m + 1)],
                    dtype=np.float64) / 4.0 ** m


def filter_line(f, axis, sigma):
    """One pass of the filter along ``axis`` of f (a new array)."""
    fm = np.moveaxis(np.asarray(f, dtype=np.float64), axis, 0)
    n = fm.shape[0]
    out = fm.copy()
    for i in range(1, n - 1):
        m = min(i, n - 1 - i, FILTER_ORDER_HALF)
        w = filter_weights(m)
        d = sum(w[k] * fm[i - m + k] for k in range(2 * m + 1))
        out[i] = fm[i] - sigma * d
    return np.moveaxis(out, 0, axis)


def filter_state(case: Case, U, sigma=None):
    """The filter applied to every field of the state vector (x pass, then y pass)."""
    sigma = case.cfg.get("filter_sigma", 0.0) if sigma is None else sigma
    g = case.grid
    q = unpack(case.tab.ns, g.nx, g.ny, np.asarray(U, dtype=np.float64))
    out = {k: filter_line(filter_line(v, 1, sigma), 0, sigma) for k, v in q.items()}
    return pack(case.tab.ns, g.nx, g.ny, out)


# Time integrators of Sec. 3.1 besides the two-register RK3: the TVD RK3 of Shu and Osher and
# the five-stage fourth-order 2N-storage scheme of Carpenter and Kennedy (the paper cites both
# families; its text gives no coefficients, so the published ones are used).
#   TVD RK3: U1 = U0 + dt R(U0); U2 = 3/4 U0 + 1/4 (U1 + dt R(U1));
#            U^{n+1} = 1/3 U0 + 2/3 (U2 + dt R(U2)); the second register keeps U0.
#   2N schemes (RK3 above, CK RK4): dQ <- A_k dQ + dt R(U); U <- U + B_k dQ.
TVD3_W = (0.0, 3.0 / 4.0, 1.0 / 3.0)     # weight of the step's start state
TVD3_S = (1.0, 1.0 / 4.0, 2.0 / 3.0)     # weight of the Euler update of the current stage
CK4_A = (0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
         -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0)
CK4_B = (1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
         1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
         2277821191437.0 / 14882151754819.0)
RK_SCHEMES = ("rk3", "tvd3", "ck4")
RK_STAGES = {"rk3": 3, "tvd3": 3, "ck4": 5}


def rk_stage_scheme(case: Case, U, W, stage, dt, scheme):
    """One stage of `scheme`: returns (U_new, W_new, R). W is the second register (dQ of the 2N
    schemes, the step's start state of TVD RK3). After the last stage the state is filtered when
    the case sets filter_sigma > 0."""
    R = rhs(case, U)
    if scheme == "tvd3":
        if stage == 0:
            W = U
        U = TVD3_W[stage] * W + TVD3_S[stage] * (U + dt * R)
    else:
        A, B = (RK_A, RK_B) if scheme == "rk3" else (CK4_A, CK4_B)
        W = A[stage] * W + dt * R
        U = U + B[stage] * W
    if (stage == RK_STAGES[scheme] - 1 and case is not None
            and case.cfg.get("filter_sigma", 0.0) > 0.0):
        U = filter_state(case, U)
    return U, W, R


def rk_stage(case: Case, U, dQ, stage, dt):
    """One stage of the two-register RK3: returns (U_new, dQ_new, R). After the last stage the
    state is filtered when the case sets filter_sigma > 0."""
    return rk_stage_scheme(case, U, dQ, stage, dt, "rk3")


def wall_fluxes(case: Case, U):
    """Wall heat flux q_w = -K dT/dy and shear tau_w = mu du/dy at the wall (nondimensional)."""
    _, parts = rhs(case, U, return_parts=True)
    sc = case.sc
    th = parts["th"]
    K = th["k"] / (sc.Re * sc.Pr) + parts["kap_st"]
    Kw = C.icf(K, 0)[0]
    return -Kw * parts["dTdy"][0], parts["tau_xy"][0]
