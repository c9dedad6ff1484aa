"""Seeded synthetic inputs shared by the CUDA path, its tests, the bench and the oracle.

This module holds case parameters and random draws only: it performs none of the method's
arithmetic (no thermodynamics, no grid metrics, no fluxes). Both sides turn these parameters into
states with their own code.

Workloads (shapes follow the paper's cases; there is no dataset):

* ``bl_case``   -- Mach 10 flat-plate boundary layer (Table 1, Table 2 proportions), 256 x 64 cells,
  tanh wall clustering, isothermal 1000 K wall, T_inf = 350 K, p_inf = 3 kPa.
* ``sbli_case`` -- oblique-shock / boundary-layer interaction, 2048 x 256 cells, domain and
  freestream of the Mach 5.92 case of Table 3 (x 19-254, y 0-36, kappa_y = 0.15, T_inf = 1110.5 K,
  p_inf = 60967 Pa); Mach number drawn in [6, 9] and flow deflection in [8, 14] degrees from the seed;
  artificial diffusivity on; the conserved state is low-pass filtered after every RK step
  (strength 0.05 on the grid-to-grid mode).
* ``serving_requests`` -- a stream of independent boundary-layer and shock / boundary-layer
  solves for the serving path: grids from 128 x 32 to 1024 x 256, boundary layers at Mach 5-20
  with wall temperature 300-1500 K, interactions at the Mach and deflection their seed draws,
  five- or eleven-species air, seeded step counts and unit-rate exponential inter-arrival gaps
  (scaled by the caller).
* ``thermo_states`` -- independent thermochemical states: T log-uniform in [300, 15000] K,
  rho log-uniform in [1e-4, 1] kg/m^3, mass fractions Dirichlet(1); ``charged_states`` the same
  for a table with ions and electrons, Dirichlet(1) over the heavy species and the electrons that
  make each state neutral.
* ``with_species`` -- any case on the eleven-species table (ions and electrons start at zero).
* ``jet_case`` -- sonic jet from a circular orifice into a Mach 8 crossflow on a spanwise-periodic
  domain (the jet case of Sec. 4 in three dimensions): 512 x 256 x 128 cells over x 38.5-71,
  y 0-10 (cubic clustering, kappa_y = 0.15), z 0-10 (periodic, 10 jet diameters), T_inf = 600 K,
  p_inf = 49800 Pa, Re_D = 25291 (Re_inf on a_inf = Re_D / Ma); orifice centre x = 52.5, spanwise
  centre, radius and momentum ratio J in [1, 3] drawn from the seed; jet sonic at T_inf; the
  orifice edge and the plume of the initial state are smoothed over 0.3 radii and two radii of
  height (a sharper plume leaves the compact interpolations negative internal energies at its
  edge).
"""
from __future__ import annotations

import numpy as np

AIR_Y = (0.767, 0.233, 0.0, 0.0, 0.0)      # N2, O2, NO, N, O
TABLE_SPECIES = {"air5": 5, "air11": 11}


def bl_case(nx=256, ny=64, seed=0, kind="cneq"):
    """Hypersonic flat-plate boundary layer (Mach 10, Re_inf = 1e5 on a_inf)."""
    return dict(
        name=f"bl_{nx}x{ny}", kind=kind, seed=seed,
        nx=nx, ny=ny, x0=14.0, x1=86.0, y0=0.0, y1=1.6, y_stretch="tanh", y_param=2.5,
        T_inf=350.0, p_inf=3000.0, Y_inf=AIR_Y, mach=10.0, reynolds=1.0e5, prandtl_cpg=0.72,
        flow="bl", wall=1, T_wall=1000.0, delta_coef=70.0, minor_species=0.02,
        shock_deflection_deg=0.0, shock_x=0.0, shock_width=0.0,
        sponge_sigma=200.0, sponge_in=5.0, sponge_out=15.0, sponge_top_cells=max(2, (26 * ny) // 211),
        artificial_diffusivity=0, C_mu=0.002, C_beta=1.75, C_kappa=0.01, C_D=0.0,
        noise_amp=1.0e-4, dt=2.0e-4, filter_sigma=0.0, diffusion_model="ramshaw", table="air5",
    )


def sbli_case(nx=2048, ny=256, seed=0, kind="cneq"):
    """Oblique shock impinging on a hypersonic boundary layer, artificial diffusivity on."""
    rng = np.random.default_rng(seed)
    mach = float(rng.uniform(6.0, 9.0))
    deflection = float(rng.uniform(8.0, 14.0))
    return dict(
        name=f"sbli_{nx}x{ny}", kind=kind, seed=seed,
        nx=nx, ny=ny, x0=19.0, x1=254.0, y0=0.0, y1=36.0, y_stretch="cubic", y_param=0.15,
        T_inf=1110.5, p_inf=60967.0, Y_inf=AIR_Y, mach=mach, reynolds=2000.0, prandtl_cpg=0.72,
        flow="sbli", wall=1, T_wall=1500.0, delta_coef=5.0 * 4.0, minor_species=0.02,
        shock_deflection_deg=deflection, shock_x=120.0, shock_width=1.0,
        sponge_sigma=200.0, sponge_in=10.0, sponge_out=30.0, sponge_top_cells=max(2, (26 * ny) // 211),
        artificial_diffusivity=1, C_mu=0.002, C_beta=1.75, C_kappa=0.01, C_D=0.01,
        noise_amp=1.0e-4, dt=2.0e-3, filter_sigma=0.05, diffusion_model="ramshaw", table="air5",
    )


def jet_case(nx=512, ny=256, nz=128, seed=0, kind="cneq"):
    """Sonic jet in a hypersonic crossflow, spanwise periodic, artificial diffusivity on."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x3e7]))
    c = bl_case(nx, ny, seed, kind)
    c.update(
        name=f"jet_{nx}x{ny}x{nz}", nz=nz, x0=38.5, x1=71.0, y0=0.0, y1=10.0, z0=0.0, z1=10.0,
        y_stretch="cubic", y_param=0.15, T_inf=600.0, p_inf=49800.0, mach=8.0,
        reynolds=25291.0 / 8.0, T_wall=1500.0, delta_coef=20.0,
        sponge_in=1.0, sponge_out=2.0, sponge_top_cells=max(2, (20 * ny) // 500),
        artificial_diffusivity=1, C_D=0.01, dt=5.0e-4, filter_sigma=0.0,
        jet=1, jet_x=52.5, jet_z=5.0 + float(rng.uniform(-1.0, 1.0)),
        jet_radius=0.5 * float(rng.uniform(0.9, 1.1)), jet_edge=0.3,
        jet_J=float(rng.uniform(1.0, 3.0)), jet_T_ratio=1.0,
    )
    return c


def with_species(cfg, table="air11"):
    """The case on another gas table: the freestream mass fractions padded with zeros (the extra
    species of air11 are the ions and the electron)."""
    ns = TABLE_SPECIES[table]
    c = dict(cfg)
    c.update(table=table, Y_inf=tuple(cfg["Y_inf"]) + (0.0,) * (ns - len(cfg["Y_inf"])),
             name=f"{cfg['name']}_{table}")
    return c


def box_case(nx=32, ny=24, seed=0, kind="cneq"):
    """Uniform freestream in a box with far-field boundaries on all sides (no wall)."""
    c = bl_case(nx, ny, seed, kind)
    c.update(name=f"box_{nx}x{ny}", wall=0, y_stretch="tanh", minor_species=0.0, noise_amp=0.0,
             sponge_in=0.0, sponge_out=0.0)
    return c


def serving_requests(n, seed=0, steps=(500, 2000), air11=0.0):
    """n requests: (case dictionary, step count, unit-rate inter-arrival gap). Shock interactions
    take at least 128 rows and a time step of 5e-4 (a quarter of the full-size case's): on 32 rows
    (cells up to 3 high where the shock of width 1 crosses them) the solve loses positivity in its
    first step, in the oracle as in the CUDA path, and over the 500-2000 steps of the serving
    stream the interactions on 64 rows and coarse x spacing (nx <= 512) turn non-physical within
    100-1100 steps at any time step tried, while every one on 128 or 256 rows (five and eleven
    species, nx 128-1024) stays clean at 5e-4. A share `air11` of the requests runs on
    eleven-species air (drawn from a stream of its own, so the requests themselves do not depend
    on the share)."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x5e7e]))
    pick = np.random.default_rng(np.random.SeedSequence([seed, 0x11a1]))
    nxs, nys = (128, 256, 512, 1024), (32, 64, 128, 256)
    out = []
    for k in range(n):
        nx, ny = int(rng.choice(nxs)), int(rng.choice(nys))
        if rng.random() < 0.5:
            c = bl_case(nx, ny, seed=int(rng.integers(1 << 30)))
            mach = float(rng.uniform(5.0, 20.0))
            c.update(mach=mach, T_wall=float(rng.uniform(300.0, 1500.0)),
                     dt=2.0e-4 * min(1.0, 10.0 / mach))
        else:
            c = sbli_case(nx, max(ny, 128), seed=int(rng.integers(1 << 30)))
            c["dt"] = 5.0e-4
        if pick.random() < air11:
            c = with_species(c, "air11")
        c["name"] = f"req{k}_{c['name']}"
        out.append((c, int(rng.integers(steps[0], steps[1] + 1)), float(rng.exponential(1.0))))
    return out


def state_noise(n, seed):
    """Perturbation field in [-1, 1], one value per entry of the conserved state vector."""
    return np.random.default_rng(np.random.SeedSequence([seed, 0x5eed])).uniform(-1.0, 1.0, n)


def thermo_states(n, seed=0, ns=5):
    """Independent states for the thermochemistry sweep: (T, rho, Y[ns, n])."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x7e57]))
    T = np.exp(rng.uniform(np.log(300.0), np.log(15000.0), n))
    rho = np.exp(rng.uniform(np.log(1.0e-4), np.log(1.0), n))
    Y = rng.dirichlet(np.ones(ns), n).T.copy()
    return T, rho, Y


def charged_states(n, M, charge, seed=0):
    """States for a table with charged species: (T, rho, Y[ns, n]) with T and rho as in
    thermo_states, heavy-species mass fractions Dirichlet(1) and the electron mass fraction that
    makes each state neutral, M_e sum_ions Y_i / M_i (then all renormalised to sum 1). M, charge:
    the table's molar masses and charges (one negative entry, the electron)."""
    M = np.asarray(M, dtype=np.float64)
    charge = np.asarray(charge)
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x10e5]))
    T = np.exp(rng.uniform(np.log(300.0), np.log(15000.0), n))
    rho = np.exp(rng.uniform(np.log(1.0e-4), np.log(1.0), n))
    heavy = np.nonzero(charge >= 0)[0]
    ie = int(np.nonzero(charge < 0)[0][0])
    Y = np.zeros((M.size, n))
    Y[heavy] = rng.dirichlet(np.ones(heavy.size), n).T
    ions = np.nonzero(charge > 0)[0]
    Y[ie] = M[ie] * np.sum(Y[ions] / M[ions, None], axis=0)
    Y /= Y.sum(axis=0)
    return T, rho, Y
