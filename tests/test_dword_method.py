"""The double-word recurrence step of the mixed-precision line operators (dword.cuh dw_step), on
the CPU: x <- r - c x carried as an unnormalised pair of binary32 words, its high word on one
product-and-sum chain and the exact rounding errors on the low word's chain. Carried out in
exactly rounded binary32 arithmetic (each FMA one rounding of the exact a*b + c), it follows the
exact recurrence to a few 2^-48 of the recurrence's scale over hundreds of steps, for the
Thomas factors the compact operators use (|c| <= 1/3) and right-hand sides of mixed sign and
scale. The GPU parity tests of the mixed path check the compiled kernels.
"""
from fractions import Fraction

import numpy as np

f32 = np.float32


def fma32(a, b, c):
    return f32(float(Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c))))


def split(x):
    h = f32(x)
    return h, f32(x - float(h))


def dw_step(x, r, c):
    ph = f32(c[0] * x[0])
    pl = fma32(c[0], x[0], -ph)                  # c.h x.h = ph + pl exactly
    sh = f32(r[0] - ph)
    bb = f32(sh - r[0])
    sl = f32(f32(r[0] - f32(sh - bb)) + f32(-ph - bb))   # r.h - ph = sh + sl exactly
    t = f32(f32(sl - pl) + fma32(-c[1], x[0], r[1]))
    return sh, fma32(-c[0], x[1], t)


def test_recurrence_within_a_few_units_of_2_pow_minus_48():
    rng = np.random.default_rng(5)
    worst = 0.0
    for trial in range(60):
        c64 = rng.uniform(-1.0 / 3.0, 1.0 / 3.0)
        c = split(c64)
        c_exact = Fraction(float(c[0])) + Fraction(float(c[1]))
        offset = rng.normal() * 1e3 if trial % 2 else 0.0
        rs = rng.normal(size=300) * 10.0 ** rng.uniform(-3, 3) + offset
        x = (f32(0.0), f32(0.0))
        xe = Fraction(0)
        for rv in rs:
            rd = split(rv)
            x = dw_step(x, rd, c)
            xe = Fraction(float(rd[0])) + Fraction(float(rd[1])) - c_exact * xe
            got = Fraction(float(x[0])) + Fraction(float(x[1]))
            worst = max(worst, float(abs(got - xe)) / float(np.abs(rs).max()))
    assert worst < 8.0 * 2.0 ** -48, worst


def test_pair_carries_what_one_word_drops():
    """The same recurrence in plain binary32 errs by ~2^-24 of its scale; the pair does not."""
    c = split(0.3)
    x, xf, xe = (f32(0.0), f32(0.0)), f32(0.0), Fraction(0)
    c_exact = Fraction(float(c[0])) + Fraction(float(c[1]))
    for rv in np.linspace(-1.0, 1.0, 200) * np.pi:
        rd = split(rv)
        x = dw_step(x, rd, c)
        xf = f32(rd[0] - f32(c[0] * xf))
        xe = Fraction(float(rd[0])) + Fraction(float(rd[1])) - c_exact * xe
    err_pair = abs(float(Fraction(float(x[0])) + Fraction(float(x[1])) - xe))
    err_single = abs(float(Fraction(float(xf)) - xe))
    assert err_pair < 1e-13 and err_single > 1e-9, (err_pair, err_single)
