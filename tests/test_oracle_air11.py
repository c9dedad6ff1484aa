"""Pins for the oracle on eleven-species air (ions and electrons; data/air11.dat). The paper
treats five-species air only: these pin the extension's bookkeeping against invariants.

* sum_s w_s = 0, and the N, O and charge balances of the production rates vanish (Eqs. 15, 20
  and the stoichiometry of the 49 reactions, ionisation included).
* Detailed balance: at the Gibbs minimum with conserved N, O and charge (an element-potential
  solve written here, with charge as a third "element"), every reaction's net rate vanishes; a
  wrong order conversion or Delta nu for the three-body electron-impact ionisation fails it.
* Without atoms and charged species the eleven-species closure is the five-species one
  (thermodynamics, transport and production rates to rounding): every added reaction needs an
  atom, an ion or an electron.
* Electron and ion thermodynamics: c_v,e = 3/2 R / M_e; diatomic ions at 300 K have c_p/R = 7/2;
  H(298.15 K) equals each species' formation enthalpy.
* The right-hand side conserves charge: for a neutral state, sum_s q_s R_s / M_s = 0 at every
  point (convection of neutral mixtures, zero conduction current of the diffusive fluxes,
  charge-conserving sources, neutral reference state).
"""
import numpy as np
import pytest

from oracle import flow as F
from oracle import gas as G
from paper_2210_05547_gb300 import inputs as I


def _states(table11, n, seed):
    T, rho, Y = I.charged_states(n, table11.M(), table11.charge(), seed=seed)
    return T, rho, Y


def test_production_rates_conserve_mass_elements_and_charge(table11):
    T, rho, Y = _states(table11, 3000, 2)
    w = G.production_rates(table11, T, rho, Y)
    M = table11.M()[:, None]
    scale = np.max(np.abs(w), axis=0) + 1e-300
    assert np.max(np.abs(w.sum(axis=0)) / scale) < 1e-14
    mol = w / M
    mscale = np.max(np.abs(mol), axis=0) + 1e-300
    A = np.array([s.atoms for s in table11.species], dtype=float).T
    q = table11.charge()
    for row in (A[0], A[1], q):
        assert np.max(np.abs(row @ mol) / mscale) < 1e-13
    assert len(table11.reactions) == 49


def _equilibrium_with_charge(table11, T, rho, bN, bO):
    """c_s = (p_std/(R T)) exp(a_s . lambda - G_s/(R T)) with a_s = (N atoms, O atoms, charge);
    lambda minimises the convex dual sum_s c_s - b . lambda with b = (bN, bO, 0) (mol/m^3)."""
    A = np.array([list(s.atoms) + [s.charge] for s in table11.species], dtype=float)   # (ns, 3)
    g = np.array([G.species_gibbs_over_rt(s, np.array([T]))[0] for s in table11.species])
    lnP = np.log(G.P_STANDARD / (G.R_UNIV * T))
    b = np.array([bN, bO, 0.0])
    lam = np.array([(np.log(bN / 2) + g[0] - lnP) / 2, (np.log(bO / 2) + g[1] - lnP) / 2, 0.0])
    for _ in range(200):
        c = np.exp(A @ lam - g + lnP)
        grad = A.T @ c - b
        H = (A * c[:, None]).T @ A
        step = np.linalg.solve(H, -grad)
        # damped Newton on the convex dual
        t = 1.0
        phi0 = c.sum() - b @ lam
        while True:
            lt = lam + t * step
            if np.exp(A @ lt - g + lnP).sum() - b @ lt <= phi0 + 1e-4 * t * grad @ step:
                break
            t *= 0.5
        lam = lt
        if np.max(np.abs(t * step)) < 1e-13:
            break
    return np.exp(A @ lam - g + lnP)


@pytest.mark.parametrize("T,rho", [(6000.0, 0.01), (9000.0, 1e-3), (12000.0, 1e-4)])
def test_detailed_balance_with_ionisation(table11, T, rho):
    M = table11.M()
    bN = rho * 2 * 0.767 / M[0]
    bO = rho * 2 * 0.233 / M[1]
    c = _equilibrium_with_charge(table11, T, rho, bN, bO)
    assert abs(c @ table11.charge()) <= 1e-12 * c.max()
    assert c[table11.electron()] > 1e-8 * c.max()             # really ionised
    kf, _, R = G.reaction_rates(table11, np.array([T]), c[:, None])
    for ir, r in enumerate(table11.reactions):
        fwd = kf[ir, 0] * np.prod(c ** r.nu_f)
        assert abs(R[ir, 0]) <= 1e-8 * fwd, (ir, R[ir, 0], fwd)


def test_neutral_subset_is_the_five_species_closure(table, table11):
    T5, rho, Y5 = I.thermo_states(2000, seed=4)
    Y5[3:] = 0.0                                             # no atoms
    Y5 /= Y5.sum(axis=0)
    Y11 = np.zeros((11, Y5.shape[1]))
    Y11[:5] = Y5
    e = G.mixture_energy(table, T5, Y5)
    a = G.thermo_eval(table, rho, e, Y5)
    b = G.thermo_eval(table11, rho, e, Y11)
    for k in ("T", "p", "cv", "mu", "k"):
        assert np.allclose(b[k], a[k], rtol=1e-14, atol=0), k
    assert np.allclose(b["D"][:5], a["D"], rtol=1e-14, atol=0)
    assert np.allclose(b["wdot"][:5], a["wdot"], rtol=1e-13, atol=1e-300)
    assert not b["wdot"][5:].any()


def test_charged_species_thermodynamics(table11):
    names = [s.name for s in table11.species]
    e = table11.species[table11.electron()]
    T = np.array([300.0, 3000.0, 30000.0])
    assert np.allclose(G.species_molar_cv(e, T), 1.5 * G.R_UNIV, rtol=1e-15)
    for nm in ("N2+", "O2+", "NO+"):
        sp = table11.species[names.index(nm)]
        cp = G.species_molar_cv(sp, np.array([300.0]))[0] + G.R_UNIV
        assert abs(cp / G.R_UNIV - 3.5) < 0.01, nm
    for sp in table11.species:
        assert abs(G.species_molar_enthalpy(sp, np.array([298.15]))[0] - sp.hf298) < 1e-6


def test_right_hand_side_conserves_charge(table11):
    cfg = I.with_species(I.sbli_case(64, 40, seed=5))
    n = sum(a * b for _, (a, b) in F.state_layout(11, 64, 40))
    case = F.make_case(cfg, table11, I.state_noise(n, 5))
    f = F.unpack(11, 64, 40, case.U0)
    names = [s.name for s in table11.species]
    M = table11.M()
    rho = f["rho"]
    # a neutral state with ions: NO+ and O+ with their electrons, taken out of NO and O
    i_nop, i_op, i_e = names.index("NO+"), names.index("O+"), table11.electron()
    f[f"rs{i_nop}"] = 2e-3 * rho * (1.0 + 0.1 * np.sin(np.arange(rho.size).reshape(rho.shape)))
    f[f"rs{i_op}"] = 1e-3 * rho
    f[f"rs{i_e}"] = M[i_e] * (f[f"rs{i_nop}"] / M[i_nop] + f[f"rs{i_op}"] / M[i_op])
    case.U_ref = F.pack(11, 64, 40, {**F.unpack(11, 64, 40, case.U_ref),
                                     **{k: f[k] for k in (f"rs{i_nop}", f"rs{i_op}", f"rs{i_e}")}})
    U = F.pack(11, 64, 40, f)
    R = F.unpack(11, 64, 40, F.rhs(case, U))
    q = table11.charge()
    charge_rate = sum(q[s] * R[f"rs{s}"] / M[s] for s in range(1, 11))
    scale = max(np.abs(R[f"rs{s}"] / M[s]).max() for s in range(1, 11) if q[s] != 0)
    assert np.abs(charge_rate).max() <= 1e-12 * scale
    assert np.abs(R[f"rs{i_e}"]).max() > 0.0
