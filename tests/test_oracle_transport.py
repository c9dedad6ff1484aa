"""Pins for the oracle's transport properties (Sec. 2.2.1, Eqs. 19, 24).

* Wilke's rule reduces to the species value for a pure gas; Eq. (19) reduces to the binary
  coefficient in a two-species mixture.
* Sutherland's law with the constants printed in Eq. (24): at T = T_S, mu = C_1 sqrt(T_S) / 2.
* Magnitudes against handbook values for air and nitrogen (loose: the Blottner and
  Lennard-Jones fits are approximations).
"""
import numpy as np

from conftest import read_golden
from oracle import flow as F
from oracle import gas as G


def test_wilke_pure_species_limit(table):
    T = np.array([500.0, 3000.0])
    mu_s = G.species_viscosity(table, T)
    k_s = G.species_conductivity(table, T, mu_s)
    for s in range(table.ns):
        X = np.zeros((table.ns, 2))
        X[s] = 1.0
        assert np.allclose(G.wilke_mix(table, X, mu_s, mu_s), mu_s[s], rtol=1e-14)
        assert np.allclose(G.wilke_mix(table, X, mu_s, k_s), k_s[s], rtol=1e-14)


def test_averaged_diffusion_binary_limit(table):
    T = np.array([1000.0, 1000.0, 1000.0])
    p = np.array([1e4, 1e4, 1e4])
    Dbin = G.binary_diffusion(table, T, p)
    X = np.zeros((table.ns, 3))
    X[0] = [0.2, 0.5, 0.9]
    X[1] = 1.0 - X[0]
    D = G.averaged_diffusion(table, X, Dbin)
    assert np.allclose(D[0], Dbin[0, 1], rtol=1e-14)
    assert np.allclose(D[1], Dbin[1, 0], rtol=1e-14)


def test_binary_diffusion_symmetric_and_scaling(table):
    T = np.array([800.0])
    D1 = G.binary_diffusion(table, T, np.array([1e5]))
    D2 = G.binary_diffusion(table, T, np.array([2e5]))
    assert np.allclose(D1, np.swapaxes(D1, 0, 1), rtol=1e-15)
    assert np.allclose(D1, 2 * D2, rtol=1e-14)       # D ~ 1/p


def test_sutherland_constants():
    c = read_golden("paper_constants.txt")
    assert F.SUTHERLAND_C1 == c["sutherland_C1"] and F.SUTHERLAND_TS == c["sutherland_TS"]
    TS = c["sutherland_TS"]
    assert abs(F.sutherland(TS) - c["sutherland_C1"] * np.sqrt(TS) / 2) < 1e-20


def test_handbook_magnitudes(table):
    T = np.array([300.0])
    X = np.zeros((table.ns, 1))
    X[0], X[1] = 0.79, 0.21
    mu_s = G.species_viscosity(table, T)
    k_s = G.species_conductivity(table, T, mu_s)
    mu = G.wilke_mix(table, X, mu_s, mu_s)[0]
    k = G.wilke_mix(table, X, mu_s, k_s)[0]
    assert 1.75e-5 < mu < 2.05e-5          # air, 300 K: 1.85e-5 Pa s
    assert 0.024 < k < 0.029               # air, 300 K: 0.026 W/(m K)
    D = G.binary_diffusion(table, T, np.array([101325.0]))
    assert 1.8e-5 < D[0, 1, 0] < 2.3e-5    # N2-O2 at 300 K, 1 atm: about 0.2 cm^2/s
