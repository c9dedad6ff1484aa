"""Pins for the oracle's low-pass filter of the conserved state (the high-order filter that
accompanies the artificial-diffusivity shock capturing of Sec. 3.3).

* Fourier symbol: on a cosine of wavenumber theta the interior of the line is multiplied by
  1 - sigma sin^10(theta / 2), and rows at distance d < 5 from an end by 1 - sigma sin^(2d)(theta/2)
  (the closed form of the binomial difference); the grid-to-grid mode is damped by exactly 1 - sigma.
* Polynomial exactness: the interior leaves polynomials up to degree 9 unchanged, distance d up
  to degree 2d - 1 (a wrong binomial weight breaks one of these).
* The end points of every line are unchanged; a uniform state is unchanged.
"""
import numpy as np
import pytest

from oracle import flow as F
from paper_2210_05547_gb300 import inputs as I

SIGMA = 0.3


@pytest.mark.parametrize("theta", [0.3, 1.1, 2.0, 2.9, np.pi])
def test_fourier_symbol(theta):
    n = 64
    i = np.arange(n)
    f = np.cos(theta * i + 0.4)
    g = F.filter_line(f, 0, SIGMA)
    for k in range(1, n - 1):
        m = min(k, n - 1 - k, 5)
        expect = f[k] * (1.0 - SIGMA * np.sin(theta / 2.0) ** (2 * m))
        assert abs(g[k] - expect) < 1e-14, (k, m)
    assert g[0] == f[0] and g[-1] == f[-1]


def test_grid_to_grid_mode_damped_by_one_minus_sigma():
    f = (-1.0) ** np.arange(40)
    g = F.filter_line(f, 0, SIGMA)
    assert np.allclose(g[1:-1], (1.0 - SIGMA) * f[1:-1], rtol=0, atol=1e-15)


@pytest.mark.parametrize("degree", range(0, 10))
def test_polynomial_exactness(degree):
    n = 48
    rng = np.random.default_rng(degree)
    x = np.arange(n) / n
    f = np.polynomial.polynomial.polyval(x, rng.uniform(-1, 1, degree + 1))
    g = F.filter_line(f, 0, SIGMA)
    scale = np.abs(f).max()
    for k in range(1, n - 1):
        m = min(k, n - 1 - k, 5)
        if degree <= 2 * m - 1:
            assert abs(g[k] - f[k]) < 1e-12 * scale, (k, m, degree)
    if degree >= 1:
        # one degree higher than the stencil preserves is changed somewhere (the pin bites)
        k = 1
        if degree == 2:
            assert abs(g[k] - f[k]) > 1e-9 * scale


def test_weights_sum_and_symmetry():
    for m in range(1, 6):
        w = F.filter_weights(m)
        assert abs(w.sum()) < 1e-15
        assert np.array_equal(w, w[::-1])
        assert abs(np.sum(w * (-1.0) ** np.arange(-m, m + 1)) - 1.0) < 1e-15


def test_filter_state_uniform_and_separable_sawtooth(table):
    cfg = I.box_case(20, 16)
    case = F.make_case(cfg, table)
    U = case.U_ref.copy()
    q = F.unpack(5, cfg["nx"], cfg["ny"], U)
    uni = F.pack(5, cfg["nx"], cfg["ny"], {k: np.full_like(v, 1.7) for k, v in q.items()})
    assert np.allclose(F.filter_state(case, uni, SIGMA), uni, rtol=1e-15, atol=0)
    saw = {}
    for k, v in q.items():
        jj, ii = np.meshgrid(np.arange(v.shape[0]), np.arange(v.shape[1]), indexing="ij")
        saw[k] = (-1.0) ** (ii + jj)
    out = F.unpack(5, cfg["nx"], cfg["ny"], F.filter_state(case, F.pack(5, cfg["nx"], cfg["ny"], saw), SIGMA))
    for k, v in out.items():
        s = saw[k]
        assert np.allclose(v[1:-1, 1:-1], (1 - SIGMA) ** 2 * s[1:-1, 1:-1], atol=1e-15)
        # line ends: the end columns only see the y pass, the end rows only the x pass
        for c in (0, -1):
            assert np.allclose(v[1:-1, c], (1 - SIGMA) * s[1:-1, c], atol=1e-15)
            assert np.allclose(v[c, 1:-1], (1 - SIGMA) * s[c, 1:-1], atol=1e-15)
        for c in ((0, 0), (0, -1), (-1, 0), (-1, -1)):
            assert v[c] == s[c]
