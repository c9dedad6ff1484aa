"""Pins for the oracle's finite-rate chemistry (Eqs. 13-15, 20).

* sum_s w_s = 0 and conservation of N and O atoms (Eq. 20 and the stoichiometry);
* detailed balance: at the composition that minimises the Gibbs energy (found here by an
  element-potential solve and, on one tiny input, by brute-force search, neither of which uses
  K_eq), every reaction's net rate vanishes;
* a closed constant-volume, constant-energy reactor integrated to long times relaxes to that
  same equilibrium.
"""
import numpy as np
import pytest
import scipy.integrate
import scipy.optimize

from oracle import gas as G


def _atoms(table):
    return np.array([sp.atoms for sp in table.species], dtype=float).T   # (2, ns)


def test_sum_of_production_rates_and_elements(table):
    from paper_2210_05547_gb300.inputs import thermo_states
    T, rho, Y = thermo_states(3000, seed=11)
    w = G.production_rates(table, T, rho, Y)
    scale = np.max(np.abs(w), axis=0) + 1e-300
    assert np.max(np.abs(w.sum(axis=0)) / scale) < 1e-14
    A = _atoms(table)
    M = table.M()
    elem_rate = A @ (w / M[:, None])     # mol of atoms per m^3 per s
    mol_scale = np.max(np.abs(w / M[:, None]), axis=0) + 1e-300
    assert np.max(np.abs(elem_rate) / mol_scale) < 1e-13


def gibbs_equilibrium(table, T, p, b):
    """Ideal-gas equilibrium at (T, p) for element totals b = (mol N, mol O), from the element
    potentials of the Gibbs minimum: X_s = (p_std/p) exp(-g_s) a^nN_s c^nO_s with sum X = 1 and
    the N/O ratio of b. With a = exp(lambda_N), c = exp(lambda_O), sum X = 1 is a quadratic in a
    for given c; the N/O ratio is then matched by bisection on ln c. K_eq is not used."""
    names = [sp.name for sp in table.species]
    g = np.array([G.species_gibbs_over_rt(sp, np.array([T]))[0] for sp in table.species])
    k = np.exp(-g) * (G.P_STANDARD / p)
    kN2, kO2, kNO, kN, kO = (k[names.index(n)] for n in ("N2", "O2", "NO", "N", "O"))
    ratio = b[0] / b[1]

    def composition(lnc):
        c = np.exp(lnc)
        A_, B_, C_ = kN2, kN + kNO * c, kO2 * c * c + kO * c - 1.0
        a = -2.0 * C_ / (B_ + np.sqrt(B_ * B_ - 4.0 * A_ * C_))
        X = {"N2": kN2 * a * a, "O2": kO2 * c * c, "NO": kNO * a * c, "N": kN * a, "O": kO * c}
        return np.array([X[n] for n in names])

    A = _atoms(table)
    # c_max: kO2 c^2 + kO c = 1
    c_max = 2.0 / (kO + np.sqrt(kO * kO + 4.0 * kO2))
    lo, hi = np.log(c_max) - 200.0, np.log(c_max)
    for _ in range(400):
        mid = 0.5 * (lo + hi)
        X = composition(mid)
        r = (A[0] @ X) / (A[1] @ X)
        if r > ratio:
            lo = mid          # too little oxygen: raise c
        else:
            hi = mid
    X = composition(0.5 * (lo + hi))
    N = b[0] / (A[0] @ X)
    return N * X


@pytest.mark.parametrize("T,p", [(2500.0, 1e4), (4000.0, 1e5), (7000.0, 3e3)])
def test_detailed_balance_at_gibbs_equilibrium(table, T, p):
    n = gibbs_equilibrium(table, T, p, np.array([2 * 0.79, 2 * 0.21]))
    conc = n / n.sum() * p / (G.R_UNIV * T)          # mol/m^3
    kf, kb, R = G.reaction_rates(table, np.array([T]), conc[:, None])
    for ir, r in enumerate(table.reactions):
        fwd = kf[ir, 0] * np.prod(conc ** r.nu_f)
        assert abs(R[ir, 0]) <= 1e-9 * fwd, (ir, R[ir, 0], fwd)


def test_brute_force_equilibrium_tiny(table):
    """Minimise G over the three free mole numbers (NO, N, O) by nested grid zooming."""
    T, p = 4000.0, 1e5
    b = np.array([2 * 0.79, 2 * 0.21])
    g = np.array([G.species_gibbs_over_rt(sp, np.array([T]))[0] for sp in table.species])

    def gibbs(nNO, nN, nO):
        nN2 = (b[0] - nNO - nN) / 2
        nO2 = (b[1] - nNO - nO) / 2
        n = np.stack([nN2, nO2, nNO, nN, nO])
        ok = np.all(n > 0, axis=0)
        n = np.where(n > 0, n, 1.0)
        N = n.sum(axis=0)
        val = np.sum(n * (g[:, None] + np.log(n / N * p / G.P_STANDARD)), axis=0)
        return np.where(ok, val, np.inf)

    lo = np.log(np.array([1e-8, 1e-8, 1e-8]))
    hi = np.log(np.array([0.4, 1.5, 0.42]))
    best = None
    for _ in range(60):
        grids = [np.linspace(lo[d], hi[d], 21) for d in range(3)]
        A_, B_, C_ = np.meshgrid(*grids, indexing="ij")
        vals = gibbs(np.exp(A_.ravel()), np.exp(B_.ravel()), np.exp(C_.ravel()))
        k = np.argmin(vals)
        best = np.array([A_.ravel()[k], B_.ravel()[k], C_.ravel()[k]])
        width = (hi - lo) / 4
        lo, hi = best - width, best + width
    n_ref = gibbs_equilibrium(table, T, p, b)
    assert np.allclose(np.exp(best), n_ref[2:], rtol=1e-6)


def test_closed_reactor_relaxes_to_equilibrium(table):
    """d(rho Y_s)/dt = w_s at fixed rho and e reaches the Gibbs equilibrium of its final (T, p)."""
    rho = 0.05
    Y0 = np.array([0.767, 0.233, 0.0, 0.0, 0.0])
    e = G.mixture_energy(table, np.array([6000.0]), Y0[:, None])[0]
    M = table.M()

    def f(t, y):
        Y = y[:, None] / rho
        T, _ = G.temperature_from_energy(table, np.array([e]), Y)
        return G.production_rates(table, T, np.array([rho]), Y)[:, 0]

    sol = scipy.integrate.solve_ivp(f, (0.0, 1.0), rho * Y0, method="Radau", rtol=1e-10,
                                    atol=1e-14)
    Yf = sol.y[:, -1] / rho
    T, _ = G.temperature_from_energy(table, np.array([e]), Yf[:, None])
    p = rho * G.mixture_gas_constant(table, Yf[:, None])[0] * T[0]
    A = _atoms(table)
    b = A @ (Yf / M)
    n_eq = gibbs_equilibrium(table, T[0], p, b)
    X_eq = n_eq / n_eq.sum()
    X_f = (Yf / M) / np.sum(Yf / M)
    assert np.allclose(X_f, X_eq, rtol=1e-5, atol=1e-9)
