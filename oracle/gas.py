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
    charge: int = 0       # elementary charges (+1 ions, -1 the electron)


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

    def charge(self):
        return np.array([s.charge for s in self.species], dtype=np.float64)

    def heavy(self):
        """Species that take part in the mixing rules and the binary diffusion pairs: all but
        the electron (it has no Blottner or Lennard-Jones data; its diffusive flux follows from
        zero conduction current)."""
        return np.array([s.charge >= 0 for s in self.species])

    def electron(self):
        """Index of the electron, or None."""
        for i, s in enumerate(self.species):
            if s.charge < 0:
                return i
        return None


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
                                       atoms=(int(v[11]), int(v[12])),
                                       charge=int(v[13]) if len(v) > 13 else 0))
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
    phi_s = sum_r X_r [1 + sqrt(mu_s/mu_r) (M_r/M_s)^(1/4)]^2 / sqrt(8 (1 + M_s/M_r)),
    both sums over the heavy species."""
    M = tab.M()
    heavy = [s for s in range(tab.ns) if tab.heavy()[s]]
    out = np.zeros_like(X[0])
    for s in heavy:
        phi = np.zeros_like(X[0])
        for r in heavy:
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
    m_sr the reduced mass, sigma_sr the mean diameter, T* = T / sqrt(eps_s eps_r). Pairs with
    the electron are not formed (infinite here: they drop out of Eq. 19)."""
    ns = tab.ns
    heavy = tab.heavy()
    D = np.full((ns, ns) + np.shape(T), np.inf)
    for s in range(ns):
        for r in range(ns):
            if not (heavy[s] and heavy[r]):
                continue
            a, b = tab.species[s], tab.species[r]
            m_sr = (a.M * b.M / (a.M + b.M)) / N_AVOGADRO
            sigma = 0.5 * (a.lj_sigma + b.lj_sigma) * 1.0e-10
            Tstar = T / math.sqrt(a.lj_eps * b.lj_eps)
            num = 3.0 / 16.0 * np.sqrt(2.0 * math.pi * (K_BOLTZMANN * T) ** 3 / m_sr)
            D[s, r] = num / (p * math.pi * sigma ** 2 * collision_integral_diffusion(Tstar))
    return D


def averaged_diffusion(tab: GasTable, X, Dbin):
    """D_s = (1 - X_s) / sum_{r != s} X_r / D_sr (Eq. 19) over the heavy species; 0 where the
    sum vanishes. Ions diffuse ambipolarly, with twice that coefficient (electrons and ions at
    one temperature); the electron's entry is 0 (its flux follows from zero current)."""
    ns = tab.ns
    heavy = tab.heavy()
    out = np.zeros_like(X)
    for s in range(ns):
        if not heavy[s]:
            continue
        den = np.zeros_like(X[0])
        for r in range(ns):
            if r != s and heavy[r]:
                den += X[r] / Dbin[s, r]
        safe = np.where(den != 0.0, den, 1.0)
        out[s] = np.where(den != 0.0, (1.0 - X[s]) / safe, 0.0)
        if tab.species[s].charge > 0:
            out[s] = 2.0 * out[s]
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


# ---------------------------------------------------------------------------------------------
# Local thermodynamic equilibrium (Sec. 2.2.2, special cases): the composition is the one of
# minimum Gibbs energy for the element content of the mixture, a function of the thermodynamic
# state alone
# ---------------------------------------------------------------------------------------------

EQ_MAX_ITER = 100
EQ_TOL = 1.0e-11            # Newton step in the element potentials that ends the iteration
EQ_MAX_STEP = 25.0          # largest change of an element potential in one step


def element_matrix(tab: GasTable):
    """a_es: atoms of element e (N, O) in one particle of species s, shape (2, ns)."""
    return np.array([[s.atoms[e] for s in tab.species] for e in range(2)], dtype=np.float64)


def element_content(tab: GasTable, Y):
    """mol of each element per kg of mixture, b_e = sum_s a_es Y_s / M_s."""
    Y = np.asarray(Y, dtype=np.float64)
    M = tab.M().reshape((-1,) + (1,) * (Y.ndim - 1))
    return np.tensordot(element_matrix(tab), Y / M, axes=1)


def equilibrium_concentrations(tab: GasTable, T, b):
    """Composition of minimum Gibbs energy at temperature T for element totals b (mol/m^3).

    At the constrained minimum of G = sum_s n_s mu_s (element totals fixed) the chemical potential
    of each species equals the sum of the element potentials of its atoms, mu_s / (R T) =
    sum_e a_es lambda_e. With the ideal-gas chemical potential
        mu_s / (R T) = G_s / (R T) + ln(c_s R T / p_std)
    each concentration is
        c_s = (p_std / (R T)) exp(a_s . lambda - G_s / (R T)),
    and lambda follows from the element totals sum_s a_es c_s = b_e, solved by Newton's method on
    ln(sum_s a_es c_s) - ln b_e. The start is, for each element, the smallest lambda_e at which one
    species made of that element alone would hold all of it: an upper bound of the solution.
    T (n,), b (2, n). Returns c (ns, n) in mol/m^3, lambda (2, n) and a convergence mask (n,).
    """
    T = np.asarray(T, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    A = element_matrix(tab)
    g = np.stack([species_gibbs_over_rt(s, T) for s in tab.species])     # (ns, n)
    lnP = np.log(P_STANDARD / (R_UNIV * T))
    lam = np.full(b.shape, np.inf)
    for s in range(tab.ns):
        for e in range(2):
            others = [k for k in range(2) if k != e]
            if A[e, s] > 0 and all(A[k, s] == 0 for k in others):
                # a_es lambda_e - g_s + ln P = ln(b_e / a_es)
                lam[e] = np.minimum(lam[e], (np.log(b[e] / A[e, s]) + g[s] - lnP) / A[e, s])
    n = T.shape[0]
    active = np.ones(n, dtype=bool)
    for _ in range(EQ_MAX_ITER):
        if not active.any():
            break
        i = np.nonzero(active)[0]
        c = np.exp(A.T @ lam[:, i] - g[:, i] + lnP[i])                 # (ns, m)
        S = A @ c                                                       # (2, m)
        F = np.log(S) - np.log(b[:, i])
        J = np.einsum("es,js,sm->mej", A, A, c) / S.T[:, :, None]       # (m, 2, 2)
        d = -np.linalg.solve(J, F.T[:, :, None])[:, :, 0].T             # (2, m)
        d = np.clip(d, -EQ_MAX_STEP, EQ_MAX_STEP)
        lam[:, i] += d
        active[i[np.max(np.abs(d), axis=0) <= EQ_TOL]] = False
    c = np.exp(A.T @ lam - g + lnP)
    return c, lam, ~active


def equilibrium_dlnc_dT(tab: GasTable, T, c, hold):
    """d ln c_s / dT along the equilibrium at fixed density (hold="rho") or at fixed pressure
    (hold="p"), element ratios fixed.

    Differentiating c_s = (p_std/(R T)) exp(a_s . lambda - G_s/(R T)) with d(G_s/(R T))/dT =
    -H_s/(R T^2) gives d ln c_s/dT = a_s . lambda' + E_s/(R T^2), E_s = H_s - R T the molar
    internal energy. At fixed density the element totals stay fixed: sum_s a_es c_s d ln c_s/dT = 0.
    At fixed pressure they scale by a common factor, sum_s a_es c_s d ln c_s/dT = s' b_e, and the
    total concentration follows p = c_tot R T: sum_s c_s d ln c_s/dT = -c_tot / T.
    """
    T = np.asarray(T, dtype=np.float64)
    A = element_matrix(tab)
    E = np.stack([species_molar_enthalpy(s, T) - R_UNIV * T for s in tab.species])
    eps = E / (R_UNIV * T * T)                                          # (ns, n)
    n = T.shape[0]
    b = A @ c
    if hold == "rho":
        M = np.einsum("es,js,sn->nej", A, A, c)                         # (n, 2, 2)
        rhs = -np.einsum("es,sn->ne", A, c * eps)
        lam_d = np.linalg.solve(M, rhs[:, :, None])[:, :, 0].T          # (2, n)
    elif hold == "p":
        M = np.zeros((n, 3, 3))
        M[:, :2, :2] = np.einsum("es,js,sn->nej", A, A, c)
        M[:, :2, 2] = -b.T
        M[:, 2, :2] = (A @ c).T
        rhs = np.zeros((n, 3))
        rhs[:, :2] = -np.einsum("es,sn->ne", A, c * eps)
        rhs[:, 2] = -c.sum(axis=0) / T - np.sum(c * eps, axis=0)
        lam_d = np.linalg.solve(M, rhs[:, :, None])[:, :2, 0].T
    else:
        raise ValueError(hold)
    return A.T @ lam_d + eps


def equilibrium_at(tab: GasTable, T, rho, bm):
    """Equilibrium mixture at temperature T and density rho (kg/m^3) with element content bm
    (mol/kg, shape (2,) or (2, n)). Returns Y (ns, n), e (J/kg) and the equilibrium heat capacity
    c_v,eq = de/dT at fixed rho (J/(kg K))."""
    T = np.asarray(T, dtype=np.float64)
    rho = np.asarray(rho, dtype=np.float64)
    bm = np.asarray(bm, dtype=np.float64)
    b = (bm if bm.ndim == 2 else bm[:, None]) * rho[None, :]
    c, _, ok = equilibrium_concentrations(tab, T, b)
    M = tab.M()[:, None]
    Y = c * M / rho
    E = np.stack([species_molar_enthalpy(s, T) - R_UNIV * T for s in tab.species])
    Cv = np.stack([species_molar_cv(s, T) for s in tab.species])
    e = np.sum(c * E, axis=0) / rho
    dlnc = equilibrium_dlnc_dT(tab, T, c, "rho")
    cv_eq = (np.sum(c * Cv, axis=0) + np.sum(E * c * dlnc, axis=0)) / rho
    return Y, e, cv_eq, ok


def lte_temperature(tab: GasTable, rho, e, bm, T0=None):
    """Solve e_eq(T; rho) = e for T: the safeguarded Newton iteration of temperature_from_energy
    with the equilibrium energy and heat capacity at fixed density. The equilibrium energy is
    S-shaped in T (c_v,eq peaks where a molecule dissociates), where plain Newton steps can cycle
    between the two shoulders without leaving the bracket; so a Newton step is also replaced by
    bisection when |f| has not fallen below half the previous step times c_v,eq (the iteration
    does not contract). Returns (T, status)."""
    rho = np.asarray(rho, dtype=np.float64)
    e = np.asarray(e, dtype=np.float64)
    n = e.shape[0]
    T = np.full(n, 1000.0) if T0 is None else np.clip(np.asarray(T0, dtype=np.float64), T_MIN, T_MAX)
    lo = np.full(n, T_MIN)
    hi = np.full(n, T_MAX)
    status = np.zeros(n, dtype=np.int32)
    _, e_lo, _, _ = equilibrium_at(tab, lo, rho, bm)
    _, e_hi, _, _ = equilibrium_at(tab, hi, rho, bm)
    below = e <= e_lo
    above = e >= e_hi
    status[below | above] |= STATUS_T_CLAMPED
    active = ~(below | above)
    T[below] = T_MIN
    T[above] = T_MAX
    bm = np.asarray(bm, dtype=np.float64)
    dx_old = np.full(n, T_MAX - T_MIN)
    for _ in range(NEWTON_MAX_ITER):
        if not active.any():
            break
        idx = np.nonzero(active)[0]
        Ti = T[idx]
        bi = bm[:, idx] if bm.ndim == 2 else bm
        _, ei, cvi, ok = equilibrium_at(tab, Ti, rho[idx], bi)
        status[idx[~ok]] |= STATUS_NOT_CONVERGED
        f = ei - e[idx]
        hi[idx] = np.where(f > 0, Ti, hi[idx])
        lo[idx] = np.where(f <= 0, Ti, lo[idx])
        Tn = Ti - f / cvi
        done = np.abs(Tn - Ti) <= NEWTON_RTOL * Ti
        outside = ~((Tn > lo[idx]) & (Tn < hi[idx]))
        slow = np.abs(2.0 * f) > np.abs(dx_old[idx] * cvi)
        Tn = np.where((outside | slow) & ~done, 0.5 * (lo[idx] + hi[idx]), Tn)
        dx_old[idx] = np.abs(Tn - Ti)
        T[idx] = Tn
        active[idx[done]] = False
    status[active] |= STATUS_NOT_CONVERGED
    return T, status


def lte_eval(tab: GasTable, rho, e, bm, T0=None):
    """Closure of a mixture in local thermodynamic equilibrium at (rho, e) with element content bm.

    T from the equilibrium energy, the equilibrium composition at (T, rho), p = rho R_mix T, the
    mixture viscosity and frozen conductivity of that composition (Wilke), and the equilibrium
    conductivity k = k_frozen + k_reactive. The reactive part is the heat the algebraic
    diffusion of Eq. (18) carries when the mole fractions follow the equilibrium at the local
    pressure: with grad X_s = (dX_s/dT)_p grad T the diffusive heat flux sum_s h_s J_s equals
    -k_reactive grad T,
        k_reactive = (rho / M_mix) sum_s M_s D_s (dX_s/dT)_p (h_s - h),   h = sum_s Y_s h_s,
    with D_s of Eq. (19). Returns a dict of SI arrays.
    """
    rho = np.asarray(rho, dtype=np.float64)
    e = np.asarray(e, dtype=np.float64)
    bm = np.asarray(bm, dtype=np.float64)
    T, status = lte_temperature(tab, rho, e, bm, T0)
    status = status | np.where(rho > 0, 0, STATUS_NONPHYSICAL).astype(np.int32)
    Y, _, cv_eq, _ = equilibrium_at(tab, T, rho, bm)
    M = tab.M()[:, None]
    c = rho * Y / M
    Rmix = mixture_gas_constant(tab, Y)
    p = rho * Rmix * T
    cv = mixture_cv(tab, T, Y)
    X = mole_fractions(tab, Y)
    mu_s = species_viscosity(tab, T)
    k_s = species_conductivity(tab, T, mu_s)
    mu = wilke_mix(tab, X, mu_s, mu_s)
    k_f = wilke_mix(tab, X, mu_s, k_s)
    D = averaged_diffusion(tab, X, binary_diffusion(tab, T, p))
    dX = X * (equilibrium_dlnc_dT(tab, T, c, "p") + 1.0 / T)
    h_s = enthalpy_species(tab, T)
    h = np.sum(Y * h_s, axis=0)
    Mmix = 1.0 / np.sum(Y / M, axis=0)
    k_r = rho / Mmix * np.sum(M * D * dX * (h_s - h), axis=0)
    gamma = (cv + Rmix) / cv
    return dict(T=T, p=p, Y=Y, X=X, dXdT=dX, cv=cv, cv_eq=cv_eq, R=Rmix, mu=mu, k_frozen=k_f,
                k_reactive=k_r, k=k_f + k_r, D=D, a=np.sqrt(gamma * p / rho), status=status)
