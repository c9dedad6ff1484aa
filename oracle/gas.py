"""FP64 oracle: per-point thermochemistry closure of the reacting Navier-Stokes equations.

TEST INFRASTRUCTURE. Only tests/, ``__graft_entry__.smoke()`` and the CPU-baseline leg of bench.py
may import this module. The product path (the CUDA library and its binding) never calls it.

What it computes, in SI units, for each state (rho, e, Y_s) -- the work the paper hands to its
real-gas library (Sec. 3.4: "each state evaluation involves the iterative solution of nonlinear
equations"):

* mixture rules rho = sum rho_s, e = sum Y_s e_s, h = sum Y_s h_s            (Eq. 12)
* species thermodynamics from statistical mechanics (Sec. 2.2.1): rigid-rotor/harmonic-oscillator
  translational, rotational, vibrational and electronic modes, formation enthalpy at 298.15 K
* temperature from internal energy by a safeguarded Newton iteration (Sec. 3.4)
* Arrhenius forward rates k_f = C T^n exp(-T_a/T), backward rates k_b = k_f / K_eq (Sec. 2.2.1)
  with the sign of the exponent read as negative
* net rates of progress (Eq. 14) with explicit-collider elementary reactions (third-body factor 1)
* mass production rates w_s = M_s sum_r (nu''_rs - nu'_rs) R_r                (Eq. 15)
* mixture viscosity and frozen conductivity (Blottner species viscosity, Eucken species
  conductivity, Wilke mixing), binary diffusion coefficients (Chapman-Enskog with a Lennard-Jones
  collision integral), and the averaged diffusion coefficient of Eq. (19)

Everything is written straight from those definitions, vectorised over points with numpy, with no
fusion or reordering. The code shares nothing with the CUDA path; it parses the gas table itself.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Exact SI constants (2019 definitions).
K_BOLTZMANN = 1.380649e-23
N_AVOGADRO = 6.02214076e23
H_PLANCK = 6.62607015e-34
R_UNIV = K_BOLTZMANN * N_AVOGADRO          # J/(mol K)
P_STANDARD = 1.0e5                          # Pa, standard-state pressure of the Gibbs energies
T_FORMATION = 298.15                        # K, reference temperature of the formation enthalpies

# Temperature bracket of the Newton inversion and its stopping rule.
T_MIN = 50.0
T_MAX = 100000.0
NEWTON_MAX_ITER = 60
NEWTON_RTOL = 1.0e-11

STATUS_NOT_CONVERGED = 1
STATUS_T_CLAMPED = 2
STATUS_NONPHYSICAL = 4


@dataclasses.dataclass
class Species:
    name: str
    M: float              # kg/mol
    hf298: float          # J/mol
    linear: int           # 0 atom, 1 linear molecule
    theta_v: float
    theta_r: float
    symmetry: float
    blottner: tuple
    lj_sigma: float       # Angstrom
    lj_eps: float         # K
    atoms: tuple          # (N, O)
    levels: list = dataclasses.field(default_factory=list)   # [(g, theta_el)]


@dataclasses.dataclass
class Reaction:
    C: float              # SI: m^3 mol^-1 s^-1 raised to (order - 1)
    n: float
    Ta: float
    nu_f: np.ndarray      # reactant stoichiometric coefficients per species
    nu_b: np.ndarray      # product stoichiometric coefficients per species


@dataclasses.dataclass
class GasTable:
    species: list
    reactions: list

    @property
    def ns(self):
        return len(self.species)

    def M(self):
        return np.array([s.M for s in self.species])


def load_table(path) -> GasTable:
    """Parse the plain-text gas table (SPECIES / LEVEL / REACTION lines)."""
    species, reactions, raw_reactions = [], [], []
    with open(path) as fh:
        for line in fh:
            line = line.split('#', 1)[0].strip()
            if not line:
                continue
            tok = line.split()
            if tok[0] == 'SPECIES':
                v = [float(x) for x in tok[2:]]
                species.append(Species(name=tok[1], M=v[0], hf298=v[1], linear=int(v[2]),
                                       theta_v=v[3], theta_r=v[4], symmetry=v[5],
                                       blottner=(v[6], v[7], v[8]), lj_sigma=v[9], lj_eps=v[10],
                                       atoms=(int(v[11]), int(v[12]))))
            elif tok[0] == 'LEVEL':
                sp = next(s for s in species if s.name == tok[1])
                sp.levels.append((float(tok[2]), float(tok[3])))
            elif tok[0] == 'REACTION':
                raw_reactions.append(tok[1:])
    names = [s.name for s in species]
    for tok in raw_reactions:
        C_cgs, n, Ta = float(tok[0]), float(tok[1]), float(tok[2])
        assert tok[3] == ':'
        arrow = tok.index('=>')
        lhs, rhs = tok[4:arrow], tok[arrow + 1:]
        nu_f = np.zeros(len(species))
        nu_b = np.zeros(len(species))
        for nm in lhs:
            nu_f[names.index(nm)] += 1
        for nm in rhs:
            nu_b[names.index(nm)] += 1
        order = nu_f.sum()
        # cm^3/mol -> m^3/mol for each concentration factor beyond the first
        C = C_cgs * (1.0e-6) ** (order - 1)
        reactions.append(Reaction(C=C, n=n, Ta=Ta, nu_f=nu_f, nu_b=nu_b))
    return GasTable(species=species, reactions=reactions)


# ---------------------------------------------------------------------------------------------
# Species thermodynamics (per species, molar, rigid rotor / harmonic oscillator)
# ---------------------------------------------------------------------------------------------

def _electronic_moments(sp: Species, T):
    """Partition function Q_el and the Boltzmann averages <theta>, <theta^2> of the levels."""
    T = np.asarray(T, dtype=np.float64)
    Q = np.zeros_like(T)
    m1 = np.zeros_like(T)
    m2 = np.zeros_like(T)
    for g, th in sp.levels:
        w = g * np.exp(-th / T)
        Q += w
        m1 += w * th
        m2 += w * th * th
    return Q, m1 / Q, m2 / Q


def species_molar_enthalpy_sensible(sp: Species, T):
    """H(T) from 0 K without formation: (5/2)RT + rotation + vibration + electronic."""
    T = np.asarray(T, dtype=np.float64)
    H = 2.5 * T
    if sp.linear:
        H = H + T
        H = H + sp.theta_v / np.expm1(sp.theta_v / T)
    _, m1, _ = _electronic_moments(sp, T)
    H = H + m1
    return R_UNIV * H


def species_molar_enthalpy(sp: Species, T):
    """Absolute molar enthalpy: formation enthalpy at 298.15 K plus the sensible rise from there."""
    return sp.hf298 + species_molar_enthalpy_sensible(sp, T) - species_molar_enthalpy_sensible(
        sp, np.float64(T_FORMATION))


def species_molar_cv(sp: Species, T):
    T = np.asarray(T, dtype=np.float64)
    cv = np.full_like(T, 1.5)
    if sp.linear:
        x = sp.theta_v / T
        cv = cv + 1.0 + x * x * np.exp(x) / np.expm1(x) ** 2
    _, m1, m2 = _electronic_moments(sp, T)
    cv = cv + (m2 - m1 * m1) / (T * T)
    return R_UNIV * cv


def species_molar_cv_internal(sp: Species, T):
    """Internal (rotation + vibration + electronic) part of c_v, used by the Eucken conductivity."""
    return species_molar_cv(sp, T) - 1.5 * R_UNIV


def species_molar_entropy(sp: Species, T):
    """Standard-state molar entropy S(T, p_std)."""
    T = np.asarray(T, dtype=np.float64)
    m = sp.M / N_AVOGADRO
    # Sackur-Tetrode
    lam = (2.0 * math.pi * m * K_BOLTZMANN * T / H_PLANCK ** 2) ** 1.5
    S = np.log(lam * K_BOLTZMANN * T / P_STANDARD) + 2.5
    if sp.linear:
        S = S + np.log(T / (sp.symmetry * sp.theta_r)) + 1.0
        x = sp.theta_v / T
        S = S + x / np.expm1(x) - np.log(-np.expm1(-x))
    Q, m1, _ = _electronic_moments(sp, T)
    S = S + np.log(Q) + m1 / T
    return R_UNIV * S


def species_gibbs_over_rt(sp: Species, T):
    """Dimensionless standard Gibbs energy G(T, p_std) / (R T)."""
    T = np.asarray(T, dtype=np.float64)
    return species_molar_enthalpy(sp, T) / (R_UNIV * T) - species_molar_entropy(sp, T) / R_UNIV


# Per unit mass, all species stacked: arrays of shape (ns, n).

def energy_species(tab: GasTable, T):
    return np.stack([(species_molar_enthalpy(s, T) - R_UNIV * np.asarray(T)) / s.M
                     for s in tab.species])


def enthalpy_species(tab: GasTable, T):
    return np.stack([species_molar_enthalpy(s, T) / s.M for s in tab.species])


def cv_species(tab: GasTable, T):
    return np.stack([species_molar_cv(s, T) / s.M for s in tab.species])


def mixture_energy(tab: GasTable, T, Y):
    """e = sum_s Y_s e_s (Eq. 12)."""
    return np.sum(Y * energy_species(tab, T), axis=0)


def mixture_cv(tab: GasTable, T, Y):
    return np.sum(Y * cv_species(tab, T), axis=0)


def mixture_gas_constant(tab: GasTable, Y):
    return R_UNIV * np.sum(Y / tab.M()[:, None], axis=0)


# ---------------------------------------------------------------------------------------------
# Temperature inversion
# ---------------------------------------------------------------------------------------------

def temperature_from_energy(tab: GasTable, e, Y, T0=None):
    """Solve sum_s Y_s e_s(T) = e for T.

    Newton steps dT = (e - e(T)) / c_v(T), kept inside a bracket [lo, hi] that shrinks around the
    root. A Newton step whose size is at most NEWTON_RTOL * T is taken and ends the iteration (the
    error after it is of order the square of that size); any other step that would leave the open
    bracket is replaced by bisection.
    Returns (T, status).
    """
    e = np.asarray(e, dtype=np.float64)
    n = e.shape[0]
    T = np.full(n, 1000.0) if T0 is None else np.clip(np.asarray(T0, dtype=np.float64), T_MIN, T_MAX)
    lo = np.full(n, T_MIN)
    hi = np.full(n, T_MAX)
    status = np.zeros(n, dtype=np.int32)
    e_lo = mixture_energy(tab, lo, Y)
    e_hi = mixture_energy(tab, hi, Y)
    below = e <= e_lo
    above = e >= e_hi
    status[below | above] |= STATUS_T_CLAMPED
    active = ~(below | above)
    T[below] = T_MIN
    T[above] = T_MAX
    for _ in range(NEWTON_MAX_ITER):
        if not active.any():
            break
        idx = np.nonzero(active)[0]
        Ti = T[idx]
        Yi = Y[:, idx]
        f = mixture_energy(tab, Ti, Yi) - e[idx]
        cv = mixture_cv(tab, Ti, Yi)
        hi[idx] = np.where(f > 0, Ti, hi[idx])
        lo[idx] = np.where(f <= 0, Ti, lo[idx])
        Tn = Ti - f / cv
        done = np.abs(Tn - Ti) <= NEWTON_RTOL * Ti
        outside = ~((Tn > lo[idx]) & (Tn < hi[idx]))
        Tn = np.where(outside & ~done, 0.5 * (lo[idx] + hi[idx]), Tn)
        T[idx] = Tn
        active[idx[done]] = False
    status[active] |= STATUS_NOT_CONVERGED
    return T, status


# ---------------------------------------------------------------------------------------------
# Kinetics (Eqs. 13-15)
# ---------------------------------------------------------------------------------------------

def reaction_rates(tab: GasTable, T, conc):
    """Forward and backward rate constants and net rates of progress R_r (Eq. 14).

    K_eq is the concentration-based equilibrium constant
      K_c = exp(-sum_s nu_s G_s/(R T)) * (p_std/(R T))^(sum_s nu_s),  nu = nu'' - nu'.
    The backward rate is formed as exp(ln k_f - ln K_c) so that it stays finite at low T.
    Returns kf, kb, R with shape (nr, n).
    """
    T = np.asarray(T, dtype=np.float64)
    g_rt = np.stack([species_gibbs_over_rt(s, T) for s in tab.species])
    lnT = np.log(T)
    ln_pref = np.log(P_STANDARD / (R_UNIV * T))
    kf_all, kb_all, R_all = [], [], []
    for r in tab.reactions:
        nu = r.nu_b - r.nu_f
        ln_kf = np.log(r.C) + r.n * lnT - r.Ta / T
        ln_kc = -np.sum(nu[:, None] * g_rt, axis=0) + nu.sum() * ln_pref
        kf = np.exp(ln_kf)
        kb = np.exp(ln_kf - ln_kc)
        fwd = np.ones_like(T)
        bwd = np.ones_like(T)
        for s in range(tab.ns):
            for _ in range(int(r.nu_f[s])):
                fwd = fwd * conc[s]
            for _ in range(int(r.nu_b[s])):
                bwd = bwd * conc[s]
        kf_all.append(kf)
        kb_all.append(kb)
        R_all.append(kf * fwd - kb * bwd)
    return np.array(kf_all), np.array(kb_all), np.array(R_all)


def production_rates(tab: GasTable, T, rho, Y):
    """w_s = M_s sum_r (nu''_rs - nu'_rs) R_r in kg/(m^3 s) (Eq. 15)."""
    M = tab.M()
    conc = rho * Y / M[:, None]
    _, _, R = reaction_rates(tab, T, conc)
    w = np.zeros_like(Y)
    for ir, r in enumerate(tab.reactions):
        nu = r.nu_b - r.nu_f
        w += (M * nu)[:, None] * R[ir][None, :]
    return w


# ---------------------------------------------------------------------------------------------
# Transport
# ---------------------------------------------------------------------------------------------

def species_viscosity(tab: GasTable, T):
    """Blottner fit mu_s = 0.1 exp((A ln T + B) ln T + C), Pa s."""
    lnT = np.log(T)
    return np.stack([0.1 * np.exp((s.blottner[0] * lnT + s.blottner[1]) * lnT + s.blottner[2])
                     for s in tab.species])


def species_conductivity(tab: GasTable, T, mu_s):
    """Eucken: k_s = mu_s (5/2 c_v,trans + c_v,internal), per unit mass."""
    out = []
    for i, s in enumerate(tab.species):
        cv_tr = 1.5 * R_UNIV / s.M
        cv_int = species_molar_cv_internal(s, T) / s.M
        out.append(mu_s[i] * (2.5 * cv_tr + cv_int))
    return np.stack(out)


def mole_fractions(tab: GasTable, Y):
    M = tab.M()[:, None]
    return (Y / M) / np.sum(Y / M, axis=0)


def wilke_mix(tab: GasTable, X, mu_s, prop_s):
    """Wilke's rule: prop = sum_s X_s prop_s / phi_s,
    phi_s = sum_r X_r [1 + sqrt(mu_s/mu_r) (M_r/M_s)^(1/4)]^2 / sqrt(8 (1 + M_s/M_r))."""
    M = tab.M()
    ns = tab.ns
    out = np.zeros_like(X[0])
    for s in range(ns):
        phi = np.zeros_like(X[0])
        for r in range(ns):
            num = (1.0 + np.sqrt(mu_s[s] / mu_s[r]) * (M[r] / M[s]) ** 0.25) ** 2
            phi += X[r] * num / np.sqrt(8.0 * (1.0 + M[s] / M[r]))
        out += X[s] * prop_s[s] / phi
    return out


def collision_integral_diffusion(Tstar):
    """Reduced Lennard-Jones collision integral Omega^(1,1)* (Neufeld, Janzen and Aziz fit)."""
    A, B, C, D, E, F, G, H = 1.06036, 0.15610, 0.19300, 0.47635, 1.03587, 1.52996, 1.76474, 3.89411
    return A / Tstar ** B + C * np.exp(-D * Tstar) + E * np.exp(-F * Tstar) + G * np.exp(-H * Tstar)


def binary_diffusion(tab: GasTable, T, p):
    """Chapman-Enskog first approximation:
    D_sr = (3/16) sqrt(2 pi (k T)^3 / m_sr) / (p pi sigma_sr^2 Omega(T*)),
    m_sr the reduced mass, sigma_sr the mean diameter, T* = T / sqrt(eps_s eps_r)."""
    ns = tab.ns
    D = np.zeros((ns, ns) + np.shape(T))
    for s in range(ns):
        for r in range(ns):
            a, b = tab.species[s], tab.species[r]
            m_sr = (a.M * b.M / (a.M + b.M)) / N_AVOGADRO
            sigma = 0.5 * (a.lj_sigma + b.lj_sigma) * 1.0e-10
            Tstar = T / math.sqrt(a.lj_eps * b.lj_eps)
            num = 3.0 / 16.0 * np.sqrt(2.0 * math.pi * (K_BOLTZMANN * T) ** 3 / m_sr)
            D[s, r] = num / (p * math.pi * sigma ** 2 * collision_integral_diffusion(Tstar))
    return D


def averaged_diffusion(tab: GasTable, X, Dbin):
    """D_s = (1 - X_s) / sum_{r != s} X_r / D_sr (Eq. 19); 0 where the sum vanishes."""
    ns = tab.ns
    out = np.zeros_like(X)
    for s in range(ns):
        den = np.zeros_like(X[0])
        for r in range(ns):
            if r != s:
                den += X[r] / Dbin[s, r]
        safe = np.where(den != 0.0, den, 1.0)
        out[s] = np.where(den != 0.0, (1.0 - X[s]) / safe, 0.0)
    return out


# ---------------------------------------------------------------------------------------------
# The closure as one call
# ---------------------------------------------------------------------------------------------

def thermo_eval(tab: GasTable, rho, e, Y, T0=None, reactions=True):
    """Full per-point closure. rho (n,), e (n,) in J/kg, Y (ns, n). Returns a dict of SI arrays."""
    rho = np.asarray(rho, dtype=np.float64)
    e = np.asarray(e, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    T, status = temperature_from_energy(tab, e, Y, T0)
    status = status | np.where(rho > 0, 0, STATUS_NONPHYSICAL).astype(np.int32)
    Rmix = mixture_gas_constant(tab, Y)
    p = rho * Rmix * T
    cv = mixture_cv(tab, T, Y)
    h_s = enthalpy_species(tab, T)
    if reactions:
        w = production_rates(tab, T, rho, Y)
    else:
        w = np.zeros_like(Y)
    X = mole_fractions(tab, Y)
    mu_s = species_viscosity(tab, T)
    k_s = species_conductivity(tab, T, mu_s)
    mu = wilke_mix(tab, X, mu_s, mu_s)
    k = wilke_mix(tab, X, mu_s, k_s)
    Dbin = binary_diffusion(tab, T, p)
    D = averaged_diffusion(tab, X, Dbin)
    gamma = (cv + Rmix) / cv
    a = np.sqrt(gamma * p / rho)
    return dict(T=T, p=p, cv=cv, R=Rmix, h_s=h_s, wdot=w, X=X, mu=mu, k=k, D=D, a=a,
                status=status)
