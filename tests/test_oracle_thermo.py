"""Pins for the oracle's species thermodynamics and temperature inversion (Sec. 2.2.1, Eq. 12).

Each check compares the oracle with something other than itself: thermodynamic identities
(c_v = de/dT, ds/dT = c_p/T evaluated by finite differences of independent functions), textbook
limits (monatomic c_v = 3/2 R), the JANAF standard entropies, and the Newton inversion's
round trip.
"""
import numpy as np
import pytest

from conftest import read_golden
from oracle import gas as G

T_GRID = np.geomspace(200.0, 20000.0, 41)


def test_cv_is_derivative_of_energy(table):
    """c_v,s(T) must equal d e_s/dT: a dropped or mis-scaled mode in either fails."""
    h = 1e-3 * T_GRID
    e_p = G.energy_species(table, T_GRID + h)
    e_m = G.energy_species(table, T_GRID - h)
    e_p2 = G.energy_species(table, T_GRID + 2 * h)
    e_m2 = G.energy_species(table, T_GRID - 2 * h)
    fd = (8 * (e_p - e_m) - (e_p2 - e_m2)) / (12 * h)
    cv = G.cv_species(table, T_GRID)
    assert np.max(np.abs(fd - cv) / cv) < 1e-8


def test_entropy_derivative_is_cp_over_T(table):
    """dS/dT = c_p/T at constant pressure (Gibbs relation), per species."""
    for sp in table.species:
        h = 1e-3 * T_GRID
        fd = (8 * (G.species_molar_entropy(sp, T_GRID + h) - G.species_molar_entropy(sp, T_GRID - h))
              - (G.species_molar_entropy(sp, T_GRID + 2 * h)
                 - G.species_molar_entropy(sp, T_GRID - 2 * h))) / (12 * h)
        cp = G.species_molar_cv(sp, T_GRID) + G.R_UNIV
        assert np.max(np.abs(fd * T_GRID - cp) / cp) < 1e-8, sp.name


def test_enthalpy_derivative_is_cp(table):
    for sp in table.species:
        h = 1e-3 * T_GRID
        fd = (G.species_molar_enthalpy(sp, T_GRID + h)
              - G.species_molar_enthalpy(sp, T_GRID - h)) / (2 * h)
        cp = G.species_molar_cv(sp, T_GRID) + G.R_UNIV
        assert np.max(np.abs(fd - cp) / cp) < 1e-5, sp.name


def test_gibbs_is_h_minus_Ts(table):
    """G/(RT) from the oracle equals (H - T S)/(R T) assembled here from H and S."""
    for sp in table.species:
        g = G.species_gibbs_over_rt(sp, T_GRID)
        ref = (G.species_molar_enthalpy(sp, T_GRID)
               - T_GRID * G.species_molar_entropy(sp, T_GRID)) / (G.R_UNIV * T_GRID)
        assert np.allclose(g, ref, rtol=1e-13, atol=1e-12)


def test_formation_enthalpy_at_reference(table):
    """H_s(298.15 K) is the tabulated formation enthalpy (0 for N2 and O2)."""
    for sp in table.species:
        H = G.species_molar_enthalpy(sp, np.array([298.15]))[0]
        assert abs(H - sp.hf298) < 1e-9 * max(1.0, abs(sp.hf298))


def test_monatomic_and_rigid_limits(table):
    """Atoms at 300 K: c_v = 3/2 R exactly for N (first excited level at 27659 K).
    Diatomics at 300 K: c_p/R = 7/2 plus a vibrational part below 1%."""
    N = next(s for s in table.species if s.name == "N")
    cv = G.species_molar_cv(N, np.array([300.0]))[0]
    assert abs(cv / G.R_UNIV - 1.5) < 1e-14
    for name in ("N2", "O2"):
        sp = next(s for s in table.species if s.name == name)
        cp = G.species_molar_cv(sp, np.array([300.0]))[0] + G.R_UNIV
        assert 3.5 <= cp / G.R_UNIV < 3.5 * 1.01


def test_high_temperature_diatomic_limit(table):
    """Without electronic levels the diatomic c_v tends to (3/2 + 1 + 1) R as T grows."""
    sp = next(s for s in table.species if s.name == "N2")
    import copy
    bare = copy.deepcopy(sp)
    bare.levels = [(1.0, 0.0)]
    cv = G.species_molar_cv(bare, np.array([1.0e6]))[0]
    assert abs(cv / G.R_UNIV - 3.5) < 1e-6


def test_standard_entropy_against_janaf(table):
    ref = read_golden("standard_entropy_298.txt")
    for sp in table.species:
        S = G.species_molar_entropy(sp, np.array([298.15]))[0]
        # rigid-rotor / harmonic-oscillator model vs tabulated values: within 0.1 J/(mol K)
        assert abs(S - ref[sp.name]) < 0.1, (sp.name, S, ref[sp.name])


def test_newton_round_trip(table):
    from paper_2210_05547_gb300.inputs import thermo_states
    T, rho, Y = thermo_states(2000, seed=3)
    e = G.mixture_energy(table, T, Y)
    T2, status = G.temperature_from_energy(table, e, Y)
    assert not status.any()
    assert np.max(np.abs(T2 - T) / T) < 1e-13


def test_newton_independent_of_initial_guess(table):
    from paper_2210_05547_gb300.inputs import thermo_states
    T, rho, Y = thermo_states(500, seed=4)
    e = G.mixture_energy(table, T, Y)
    Ta, _ = G.temperature_from_energy(table, e, Y, T0=np.full_like(T, 60.0))
    Tb, _ = G.temperature_from_energy(table, e, Y, T0=np.full_like(T, 90000.0))
    # floor: rounding of sum Y_s e_s with formation energies up to ~3e7 J/kg against c_v T
    assert np.max(np.abs(Ta - Tb) / Ta) < 1e-13


def test_newton_flags_out_of_range(table):
    Y = np.array([[1.0], [0.0], [0.0], [0.0], [0.0]])
    e_low = G.mixture_energy(table, np.array([G.T_MIN]), Y) - 1e5
    T, status = G.temperature_from_energy(table, e_low, Y)
    assert status[0] & G.STATUS_T_CLAMPED and T[0] == G.T_MIN


def test_equation_of_state_and_sound_speed(table):
    """p = rho R_u T sum Y/M; frozen sound speed of cold air near the textbook 374 m/s at 350 K."""
    Y = np.array([[0.767], [0.233], [0.0], [0.0], [0.0]])
    T = np.array([350.0])
    rho = np.array([0.03])
    out = G.thermo_eval(table, rho, G.mixture_energy(table, T, Y), Y)
    p_ref = 0.03 * 8.314462618 * 350.0 * (0.767 / 0.0280134 + 0.233 / 0.0319988)
    assert abs(out["p"][0] / p_ref - 1.0) < 1e-9      # R_u = N_A k_B = 8.314462618... J/(mol K)
    assert 370.0 < out["a"][0] < 380.0
