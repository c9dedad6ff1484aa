"""Pins of the oracle's artificial diffusivity (Sec. 3.3 and the localized-artificial-diffusivity
form of the papers it cites): the fourth index difference, the nine-point truncated Gaussian
filter, the Ducros switch and the four diffusivities built from them.

Each assertion names the plausible mistake it catches. Nothing here compares the oracle with
itself: the expected values are closed forms (finite differences of polynomials, sums of the
published filter weights as fractions, Fourier responses) or orders of convergence."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import flow as F

CFG = {"C_mu": 0.002, "C_beta": 1.75, "C_kappa": 0.01, "C_D": 0.01}
WEIGHTS = (Fraction(3565, 10368), Fraction(3091, 12960), Fraction(1997, 25920),
           Fraction(149, 12960), Fraction(107, 103680))


# ---------------------------------------------------------------------------------------------
# delta4: (1, -4, 6, -4, 1), the two rows nearest each end reuse the nearest full stencil
# ---------------------------------------------------------------------------------------------

@pytest.mark.parametrize("axis", [0, 1])
def test_delta4_annihilates_cubics_at_every_row(axis):
    """A fourth difference vanishes on every cubic, end rows included (a wrong coefficient, or an
    end row that falls back to a shorter stencil, leaves a non-zero result)."""
    i = np.arange(23, dtype=np.float64)
    for coef in ([3.0, -2.0, 5.0, 1.0], [0.0, 0.0, 0.0, 7.0], [1.0, 1.0, 1.0, 0.0]):
        f1 = coef[0] + coef[1] * i + coef[2] * i ** 2 + coef[3] * i ** 3
        f = np.stack([f1, 2.0 * f1, -f1]) if axis == 1 else np.stack([f1, 2.0 * f1, -f1], axis=1)
        assert np.array_equal(F.delta4(f, axis), np.zeros_like(f))


@pytest.mark.parametrize("axis", [0, 1])
def test_delta4_of_quartic_is_24_at_every_row(axis):
    """The fourth difference of i^4 on unit spacing is 4! = 24 at every row (interior and the two
    end rows on each side): a stencil off by a factor, a sign flip or an end row that is left at
    zero all change it. The other axis is left alone (a transposed axis gives 0 here)."""
    i = np.arange(17, dtype=np.float64)
    f1 = i ** 4
    f = np.stack([f1] * 6) if axis == 1 else np.stack([f1] * 6, axis=1)
    d = F.delta4(f, axis)
    assert np.array_equal(d, np.full_like(f, 24.0))
    assert np.array_equal(F.delta4(f, 1 - axis), np.zeros_like(f))


def test_delta4_end_rows_reuse_the_nearest_full_stencil():
    """Rows 0, 1 take the stencil centred on row 2 and rows n-2, n-1 the one centred on n-3, so an
    i^5 field (whose fourth difference is 120 i) gives 120 * 2 at the first two rows."""
    i = np.arange(12, dtype=np.float64)
    d = F.delta4(i ** 5, 0)
    centre = np.clip(np.arange(12), 2, 9)
    assert np.array_equal(d, 120.0 * centre)


# ---------------------------------------------------------------------------------------------
# gauss9: nine-point truncated Gaussian, clamped indices at the ends
# ---------------------------------------------------------------------------------------------

def test_gauss9_weights_are_the_published_fractions():
    """The oracle's weights equal the published fractions; they sum to one (w0 + 2 sum w_d), the
    grid-to-grid mode is removed exactly (w0 + 2 sum (-1)^d w_d = 0) and the kernel's second
    moment 2 sum d^2 w_d is 4/3. A typo in any one weight breaks at least one of the three."""
    for got, want in zip(F.GAUSS9, WEIGHTS):
        assert got == float(want)
    assert WEIGHTS[0] + 2 * sum(WEIGHTS[1:]) == 1
    assert WEIGHTS[0] + 2 * sum((-1) ** d * WEIGHTS[d] for d in range(1, 5)) == 0
    assert 2 * sum(d * d * WEIGHTS[d] for d in range(1, 5)) == Fraction(4, 3)


@pytest.mark.parametrize("axis", [0, 1])
def test_gauss9_constants_pass_and_grid_mode_vanishes(axis):
    """Constants pass unchanged at every row (clamped ends included; dropping the clamp or a
    weight changes the ends); the (-1)^i mode vanishes at rows 4 .. n-5 where the stencil fits;
    linear data pass unchanged there (the kernel is symmetric)."""
    n = 21
    i = np.arange(n, dtype=np.float64)
    shape_line = (lambda v: np.stack([v, v, v])) if axis == 1 else (lambda v: np.stack([v, v, v], 1))
    c = shape_line(np.full(n, 3.25))
    assert np.allclose(F.gauss9(c, axis), c, rtol=2e-16, atol=0.0)
    alt = shape_line((-1.0) ** i)
    out = F.gauss9(alt, axis)
    inner = out[:, 4:n - 4] if axis == 1 else out[4:n - 4, :]
    assert np.abs(inner).max() <= 1e-16
    lin = shape_line(0.5 + 2.0 * i)
    outl = F.gauss9(lin, axis)
    sl = (slice(None), slice(4, n - 4)) if axis == 1 else (slice(4, n - 4), slice(None))
    assert np.allclose(outl[sl], lin[sl], rtol=1e-15, atol=0.0)


def test_gauss9_second_moment_on_quadratic():
    """On f = i^2 the filter adds its second moment, 4/3, at interior rows (a wrong weight, or the
    weights applied at the wrong distances, changes the added constant)."""
    i = np.arange(30, dtype=np.float64)
    out = F.gauss9(i ** 2, 0)
    assert np.allclose(out[4:-4] - (i ** 2)[4:-4], 4.0 / 3.0, rtol=0.0, atol=1e-12)


def test_filter2_filters_both_directions():
    """filter2 removes the grid-to-grid mode along x and along y (a filter over one direction
    only leaves one of them)."""
    ny, nx = 18, 20
    j, i = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    for f in ((-1.0) ** i, (-1.0) ** j):
        out = F.filter2(f.astype(np.float64))
        assert np.abs(out[4:-4, 4:-4]).max() <= 1e-16


# ---------------------------------------------------------------------------------------------
# Ducros switch and the four diffusivities
# ---------------------------------------------------------------------------------------------

def test_ducros_switch_rotation_compression_expansion():
    """Pure rotation (div u = 0, omega != 0) gives 0, pure compression (omega = 0, div u < 0)
    gives 1, expansion (div u > 0) gives 0 (a flipped Heaviside condition swaps the last two; a
    missing square gives values other than 0 and 1)."""
    om = np.array([2.0, -3.0, 0.5])
    assert np.array_equal(F.ducros(np.zeros(3), om), np.zeros(3))
    div = np.array([-1.0, -0.25, -40.0])
    assert np.allclose(F.ducros(div, np.zeros(3)), 1.0, rtol=1e-15, atol=0.0)
    assert np.array_equal(F.ducros(-div, np.zeros(3)), np.zeros(3))
    # equal strengths: one half
    assert np.allclose(F.ducros(np.array([-2.0]), np.array([2.0])), 0.5, rtol=1e-15)


def _fields(ny, nx, dx, dy, u, v, e, Y, rho=None):
    """Centre fields of analytic velocity, energy and mass fractions on a uniform grid; the
    velocity gradients are the exact derivatives of u and v (functions of (x, y) returning the
    value and both derivatives)."""
    y = (np.arange(ny) + 0.5)[:, None] * dy
    x = (np.arange(nx) + 0.5)[None, :] * dx
    uu, ux, uy = u(x, y)
    vv, vx, vy = v(x, y)
    shape = (ny, nx)
    b = lambda a: np.broadcast_to(np.asarray(a, dtype=np.float64), shape).copy()
    rho = b(1.3 if rho is None else rho)
    a = b(2.1)
    T = b(1.7)
    return dict(rho=rho, a=a, T=T, e=b(e(x, y)), Y=np.stack([b(f(x, y)) for f in Y]),
                dudx=b(ux), dvdy=b(vy), dudy_c=b(uy), dvdx_c=b(vx), dx=b(dx), dy=b(dy))


def _ad(fl):
    return F.artificial_diffusivity(CFG, fl["rho"], fl["a"], fl["T"], fl["e"], fl["Y"],
                                    fl["dudx"], fl["dvdy"], fl["dudy_c"], fl["dvdx_c"],
                                    fl["dx"], fl["dy"])


def test_diffusivities_vanish_on_linear_fields():
    """Linear velocity (constant strain and divergence), linear energy and mass fractions give
    mu* = beta* = kappa* = D* = 0 up to rounding of the constant strain; the same magnitudes with
    a quartic component give clearly non-zero values (a sensor built from a second difference,
    or from the field instead of its fourth difference, does not vanish on linear fields)."""
    dx, dy = 0.05, 0.03
    lin = _fields(24, 26, dx, dy,
                  u=lambda x, y: (-0.8 * x + 0.3 * y, -0.8, 0.3),
                  v=lambda x, y: (0.2 * x - 0.5 * y, 0.2, -0.5),
                  e=lambda x, y: 2.0 + 0.7 * x - 0.4 * y,
                  Y=[lambda x, y: 0.2 + 0.1 * x + 0.05 * y, lambda x, y: 0.3 - 0.02 * x])
    out = _ad(lin)
    for k, arr in zip(("mu", "beta", "kappa", "D"), out):
        assert np.abs(arr).max() <= 1e-15, k
    quart = _fields(24, 26, dx, dy,
                    u=lambda x, y: (-0.8 * x - x ** 5, -0.8 - 5 * x ** 4, 0.0 * x),
                    v=lambda x, y: (-0.5 * y - y ** 5, 0.0 * y, -0.5 - 5 * y ** 4),
                    e=lambda x, y: 2.0 + x ** 5 + y ** 5,
                    Y=[lambda x, y: 0.2 + x ** 5, lambda x, y: 0.3 + y ** 5])
    outq = _ad(quart)
    for k, arr in zip(("mu", "beta", "kappa", "D"), outq):
        assert np.abs(arr).max() > 1e-9, k


def _centre_value(n, f_of_xy, which):
    """One diffusivity at the physical point (0.5, 0.5) of the unit square on an n x n grid."""
    d = 1.0 / n
    fl = _fields(n, n, d, d, **f_of_xy)
    arr = _ad(fl)[which]
    if which == 3:
        arr = arr[0]
    # (0.5, 0.5) lies on the corner of the four middle cells: average them
    m = n // 2
    return float(arr[m - 1:m + 1, m - 1:m + 1].mean())


SMOOTH = dict(u=lambda x, y: (np.sin(2 * x) + 0.3 * np.cos(y), 2 * np.cos(2 * x), -0.3 * np.sin(y)),
              v=lambda x, y: (np.cos(3 * y) - 0.2 * np.sin(x), -0.2 * np.cos(x), -3 * np.sin(3 * y)),
              e=lambda x, y: 2.0 + np.sin(2 * x) + np.cos(1.5 * y),
              Y=[lambda x, y: 0.2 + 0.1 * np.sin(3 * x) * np.cos(y)])


@pytest.mark.parametrize("which,order", [(0, 6), (1, 6), (2, 5), (3, 5)],
                         ids=["mu_star", "beta_star", "kappa_star", "D_star"])
def test_diffusivities_scale_with_grid_size(which, order):
    """On fixed smooth fields the fourth index difference is O(d^4), so mu* and beta* (times d^2)
    fall as d^6 and kappa*, D* (times d) as d^5 under grid halving: the ratio of successive
    values approaches 2^6 or 2^5 (a d instead of d^2, or d^2 instead of d, moves the order by
    one; a missing metric factor by two)."""
    v = [_centre_value(n, SMOOTH, which) for n in (64, 128, 256)]
    assert all(x > 0 for x in v)
    r1, r2 = v[0] / v[1], v[1] / v[2]
    assert abs(np.log2(r2) - order) < 0.05, (r1, r2)
    assert abs(np.log2(r2) - order) <= abs(np.log2(r1) - order) + 1e-3


def test_x_and_y_contributions_sum_inside_the_absolute_value():
    """mu* takes |d4_x(S) dx^2 + d4_y(S) dy^2|: for S varying along x only, and then along y
    only with the same profile and spacing, mu* is the transpose (a direction dropped or its
    metric swapped breaks the symmetry)."""
    n, d = 32, 0.04
    fx = _fields(n, n, d, d, u=lambda x, y: (x ** 4 * 0.0 + np.sin(3 * x), 3 * np.cos(3 * x), 0.0 * y),
                 v=lambda x, y: (0.0 * x, 0.0 * x, 0.0 * y),
                 e=lambda x, y: np.cos(2 * x), Y=[lambda x, y: 0.1 + 0.0 * x])
    fy = _fields(n, n, d, d, u=lambda x, y: (0.0 * x, 0.0 * x, 0.0 * y),
                 v=lambda x, y: (np.sin(3 * y), 0.0 * y, 3 * np.cos(3 * y)),
                 e=lambda x, y: np.cos(2 * y), Y=[lambda x, y: 0.1 + 0.0 * y])
    ax, ay = _ad(fx), _ad(fy)
    for k in (0, 1, 2):
        assert np.abs(ax[k]).max() > 0
        assert np.allclose(ax[k], ay[k].T, rtol=1e-13, atol=1e-300), k


def test_constants_enter_linearly():
    """Each diffusivity is proportional to its own constant and to rho (mu*, beta*, kappa*) or
    the sound speed (kappa*, D*): doubling C_mu doubles mu* only; doubling a doubles kappa* and
    D*; doubling rho doubles mu*, beta*, kappa* and leaves D* unchanged."""
    n, d = 24, 0.05
    base = _fields(n, n, d, d, **SMOOTH)
    ref = _ad(base)
    cfg2 = dict(CFG, C_mu=2 * CFG["C_mu"])
    out = F.artificial_diffusivity(cfg2, base["rho"], base["a"], base["T"], base["e"], base["Y"],
                                   base["dudx"], base["dvdy"], base["dudy_c"], base["dvdx_c"],
                                   base["dx"], base["dy"])
    assert np.allclose(out[0], 2 * ref[0], rtol=1e-14)
    for k in (1, 2, 3):
        assert np.array_equal(out[k], ref[k])
    fa = dict(base, a=2 * base["a"])
    oa = _ad(fa)
    assert np.allclose(oa[2], 2 * ref[2], rtol=1e-14) and np.allclose(oa[3], 2 * ref[3], rtol=1e-14)
    assert np.array_equal(oa[0], ref[0]) and np.array_equal(oa[1], ref[1])
    fr = dict(base, rho=2 * base["rho"])
    orr = _ad(fr)
    for k in (0, 1, 2):
        assert np.allclose(orr[k], 2 * ref[k], rtol=1e-14), k
    assert np.array_equal(orr[3], ref[3])


def test_each_direction_takes_its_own_cell_size():
    """Data varying along y only: mu* and beta* scale with dy^2 and kappa*, D* with dy, and none
    depends on dx (and the same along x with the roles swapped). A cell size of the wrong
    direction, or dx^2 where dx is due, fails the ratios."""
    n = 20
    j, i = np.meshgrid(np.arange(n, dtype=np.float64), np.arange(n, dtype=np.float64), indexing="ij")
    for along_y in (True, False):
        s = j if along_y else i
        prof = np.sin(0.7 * s) + 0.1 * s ** 2
        fl = dict(rho=np.full((n, n), 1.3), a=np.full((n, n), 2.1), T=np.full((n, n), 1.7),
                  e=2.0 + prof, Y=np.stack([0.2 + 0.05 * prof]),
                  dudx=np.zeros((n, n)) if along_y else -0.5 - 0.3 * prof,
                  dvdy=-0.5 - 0.3 * prof if along_y else np.zeros((n, n)),
                  dudy_c=np.zeros((n, n)), dvdx_c=np.zeros((n, n)))

        def run(dx, dy):
            return F.artificial_diffusivity(CFG, fl["rho"], fl["a"], fl["T"], fl["e"], fl["Y"],
                                            fl["dudx"], fl["dvdy"], fl["dudy_c"], fl["dvdx_c"],
                                            np.full((n, n), dx), np.full((n, n), dy))
        base = run(0.01, 0.01)
        other = run(0.04, 0.01) if along_y else run(0.01, 0.04)
        own = run(0.01, 0.02) if along_y else run(0.02, 0.01)
        for k, power in ((0, 2), (1, 2), (2, 1), (3, 1)):
            b = base[k]
            assert np.abs(b).max() > 0, k
            assert np.allclose(other[k], b, rtol=1e-12, atol=0.0), (along_y, k)
            assert np.allclose(own[k], 2.0 ** power * b, rtol=1e-12, atol=0.0), (along_y, k)
