"""Pin of the magnitude and units of the forward and backward rates (Eqs. 13-15).

Sum rules, element conservation, detailed balance and the closed reactor all hold for any
forward-rate constant, so they cannot see a wrong unit conversion of Park's constants (printed in
cm^3 mol^-1 s^-1 per extra reactant). This test computes the mass production rates a second way,
entirely in the units the rate constants are printed in: concentrations in mol/cm^3, k_f in
(cm^3/mol)^(order-1)/s straight from the table's REACTION lines, the equilibrium constant with
the standard concentration p_std/(R_u T) in mol/cm^3 (p_std = 1e6 dyn/cm^2, R_u in erg/(mol K)),
rates of progress in mol/(cm^3 s) and w_s in g/(cm^3 s); it converts to kg/(m^3 s) once at the
end. A conversion that is off by one order (1e-6^order instead of 1e-6^(order-1)), applied to
the backward rates' extra product, or forgotten, changes the result by factors of 1e6."""
import os

import numpy as np
import pytest

from oracle import gas as G

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
R_ERG = 1.380649e-16 * 6.02214076e23   # erg / (mol K): k_B in erg/K times N_A (exact SI values)
P_STD_CGS = 1.0e6              # dyn / cm^2 (1 bar)


def _raw_table(path):
    """Species names and molar masses (g/mol), and the REACTION lines as printed."""
    names, M_g, reactions = [], [], []
    with open(path) as fh:
        for line in fh:
            tok = line.split("#", 1)[0].split()
            if not tok:
                continue
            if tok[0] == "SPECIES":
                names.append(tok[1])
                M_g.append(float(tok[2]) * 1000.0)
            elif tok[0] == "REACTION":
                arrow = tok.index("=>")
                reactions.append((float(tok[1]), float(tok[2]), float(tok[3]),
                                  tok[5:arrow], tok[arrow + 1:]))
    return names, np.array(M_g), reactions


def _wdot_cgs(table, path, T, rho_si, Y):
    names, M_g, reactions = _raw_table(path)
    rho_cgs = rho_si * 1.0e-3                           # g / cm^3
    conc = rho_cgs * Y / M_g[:, None]                   # mol / cm^3
    g_rt = np.stack([G.species_gibbs_over_rt(sp, T) for sp in table.species])
    c_std = P_STD_CGS / (R_ERG * T)                     # mol / cm^3
    w = np.zeros_like(Y)
    gross = np.zeros_like(Y)
    for C_cgs, n, Ta, lhs, rhs in reactions:
        nu_f = np.zeros(len(names))
        nu_b = np.zeros(len(names))
        for nm in lhs:
            nu_f[names.index(nm)] += 1
        for nm in rhs:
            nu_b[names.index(nm)] += 1
        nu = nu_b - nu_f
        kf = C_cgs * T ** n * np.exp(-Ta / T)           # (cm^3/mol)^(order-1) / s
        Kc = np.exp(-(nu[:, None] * g_rt).sum(axis=0)) * c_std ** nu.sum()
        fwd = np.prod([conc[s] ** nu_f[s] for s in range(len(names))], axis=0)
        bwd = np.prod([conc[s] ** nu_b[s] for s in range(len(names))], axis=0)
        R = kf * fwd - kf / Kc * bwd                    # mol / (cm^3 s)
        w += (M_g * nu)[:, None] * R[None, :]           # g / (cm^3 s)
        gross += np.abs(M_g * nu)[:, None] * (kf * fwd + kf / Kc * bwd)[None, :]
    return w * 1.0e3, gross * 1.0e3                     # kg / (m^3 s)


@pytest.mark.parametrize("which", ["air5", "air11"])
def test_production_rates_in_park_units(table, table11, which):
    from paper_2210_05547_gb300.inputs import charged_states, thermo_states
    tab = table if which == "air5" else table11
    path = os.path.join(ROOT, "paper_2210_05547_gb300", "data", f"{which}.dat")
    if which == "air5":
        T, rho, Y = thermo_states(400, seed=21)
    else:
        # ions and electrons present: the ionisation reactions (three-body electron impact
        # included) take part
        T, rho, Y = charged_states(400, tab.M(), [sp.charge for sp in tab.species], seed=21)
    sel = (T > 1500.0) & (T < 12000.0)
    T, rho, Y = T[sel], rho[sel], Y[:, sel]
    want, gross = _wdot_cgs(tab, path, T, rho, Y)
    got = G.production_rates(tab, T, rho, Y)
    for s in range(tab.ns):
        # Both sides exponentiate arguments of up to a few hundred (a few hundred eps apart in
        # each forward and backward term), and a net rate can be a small difference of the two
        # (fast ionisation near its balance): the floor is set by the gross rate of the species,
        # sum_r |M_s nu_rs| (forward + backward), not by the net rate.
        scale = gross[s].max()
        if scale == 0.0:
            assert np.abs(got[s]).max() == 0.0
            continue
        assert np.abs(got[s] - want[s]).max() <= 1e-12 * scale, (which, s)
    # and pointwise where the rate is not a cancellation of forward and backward terms
    big = np.abs(want) > 1e-6 * np.abs(want).max(axis=1, keepdims=True)
    rel = np.abs(got - want)[big] / np.abs(want)[big]
    assert rel.max() < 1e-9
