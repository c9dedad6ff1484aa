"""Pins for the oracle's Stefan-Maxwell diffusion (Eq. 17).

* With one binary coefficient for every pair the Stefan-Maxwell fluxes equal the algebraic
  fluxes of Eq. (18) (with the gradient of X, Eq. 16) exactly: the closed form of the system.
* The fluxes sum to zero, and the entropy production they imply is never negative:
  sum_s V_s . d_s = -sum_{s<i} X_s X_i (V_s - V_i)^2 / D_si <= 0, with V_s = J_s / (rho Y_s).
* A species of zero mole fraction gets the flux its own row gives in closed form,
  J_s = -rho (M_s / Mbar) d_s / sum_{i != s} X_i / D_si.
* Binary mixtures reduce to Fick's law: test_pde_consistency_binary_diffusion (test_oracle_flow)
  runs with both diffusion models.
"""
import numpy as np

from oracle import flow as F


def _random(table, n=400, seed=0, zero=None):
    rng = np.random.default_rng(seed)
    Y = rng.dirichlet(np.ones(5), n).T
    Y[0] += 1.0                                      # the omitted species dominates, as in air
    Y /= Y.sum(axis=0)
    if zero is not None:
        Y[zero] = 0.0
        Y /= Y.sum(axis=0)
    rho = rng.uniform(0.2, 2.0, n)
    dX = rng.normal(size=(5, n))
    dX -= dX.mean(axis=0)                            # sum_s grad X_s = 0
    D = rng.uniform(0.5, 3.0, (5, 5, n))
    D = 0.5 * (D + D.transpose(1, 0, 2))
    return rho, Y, dX, D


def test_equal_coefficients_give_the_algebraic_flux(table):
    rho, Y, dX, _ = _random(table, seed=1)
    Dc = 1.7
    D = np.full((5, 5, rho.size), Dc)
    J = F.stefan_maxwell_fluxes(table, rho, Y, dX, D)
    M = table.M()[:, None]
    Mbar = 1.0 / np.sum(Y / M, axis=0)
    G = rho * M / Mbar * Dc                          # rho (M_s / Mbar) D_s with D_s = D
    g = G * dX
    ram = -(g - Y * g.sum(axis=0))
    assert np.max(np.abs(J - ram)) < 1e-12 * np.max(np.abs(ram))


def test_fluxes_sum_to_zero_and_dissipate(table):
    rho, Y, dX, D = _random(table, seed=2)
    J = F.stefan_maxwell_fluxes(table, rho, Y, dX, D)
    assert np.max(np.abs(J.sum(axis=0))) < 1e-13 * np.max(np.abs(J))
    V = J / (rho * Y)
    production = np.sum(V * dX, axis=0)
    assert np.all(production <= 1e-12 * np.max(np.abs(V * dX)))
    assert np.min(production) < 0.0


def test_trace_species_row(table):
    rho, Y, dX, D = _random(table, seed=3, zero=3)
    J = F.stefan_maxwell_fluxes(table, rho, Y, dX, D)
    M = table.M()
    Mbar = 1.0 / np.sum(Y / M[:, None], axis=0)
    X = Y / M[:, None] * Mbar
    s = 3
    den = sum(X[i] / D[s, i] for i in range(5) if i != s)
    expect = -rho * (M[s] / Mbar) * dX[s] / den
    assert np.max(np.abs(J[s] - expect)) < 1e-12 * np.max(np.abs(expect))
