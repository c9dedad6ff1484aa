"""The constant tables of the closure's table-driven exponential and logarithm (fp64_fast.cuh), on
the CPU: the committed headers are what their generators write, the tables hold what their
comments say, and the two methods (Tang's exponential, ACM TOMS 15(2) 1989; Tang's logarithm in
reciprocal form, ACM TOMS 16(4) 1990) reach their stated accuracy when their steps are carried
out in exactly rounded binary64 arithmetic with these tables. The GPU test
(test_gpu_fp64_fast.py) checks the compiled functions themselves.

The steps below follow the methods as published. Each fused multiply-add is one rounding of the
exact a*b + c; the reference values come from 40-digit decimal arithmetic.
"""
import decimal
import importlib.util
import math
import os
from fractions import Fraction

import numpy as np

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_2210_05547_gb300", "csrc")
D = decimal.Decimal
decimal.getcontext().prec = 40


def _load(name):
    spec = importlib.util.spec_from_file_location(name, os.path.join(CSRC, name + ".py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def fma(a, b, c):
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def ulps(got, exact):
    """|got - exact| in units of the last place of the binary64 nearest to exact."""
    ref = float(exact)
    return float(abs(D(got) - exact) / D(math.ulp(ref)))


def test_headers_are_the_generators_output():
    for gen, header in (("gen_exp_table", "exp_table.h"), ("gen_log_table", "log_table.h")):
        with open(os.path.join(CSRC, header)) as fh:
            assert fh.read() == _load(gen).render(), header


def test_exp_table_entries():
    table, c_hi, c_lo, inv = _load("gen_exp_table").tables()
    ln2 = D(2).ln()
    for j, t in enumerate(table):
        exact = (D(j) / 256 * ln2).exp()
        assert ulps(t, exact) <= 0.5, j
    # C_HI has 33 significant bits, so n C_HI is exact for |n| < 2^20; C_HI + C_LO = ln2/256
    assert Fraction(c_hi).numerator.bit_length() <= 33
    assert abs(D(c_hi) + D(c_lo) - ln2 / 256) < D(2) ** -90
    assert abs(D(inv) - 256 / ln2) / (256 / ln2) < D(2) ** -24


def test_log_table_entries():
    rows, ln2_hi, ln2_lo = _load("gen_log_table").tables()
    for j, (inv, t_hi, t_lo) in enumerate(rows):
        c = 1 + (D(j) + D("0.5")) / 128
        assert ulps(inv, 1 / c) <= 0.5, j
        assert abs(D(t_hi) + D(t_lo) + D(inv).ln()) < D(2) ** -100, j
    assert Fraction(ln2_hi).numerator.bit_length() <= 42     # k LN2_HI exact for |k| < 2^11
    assert abs(D(ln2_hi) + D(ln2_lo) - D(2).ln()) < D(2) ** -95


def _tang_exp(x, table, c_hi, c_lo, inv):
    n = int(np.rint(np.float32(np.float32(x) * np.float32(inv))))
    r = fma(-n, c_hi, x)
    r = fma(-n, c_lo, r)
    r2 = r * r
    c = fma(r, 1.0 / 24.0, 1.0 / 6.0)
    c = fma(r, c, 0.5)
    p = fma(r2, c, r)
    tj = table[n % 256]
    y = fma(tj, p, tj)
    return math.ldexp(y, n // 256)


def _table_log(x, rows, ln2_hi, ln2_lo):
    m, e = math.frexp(x)              # x = m 2^e, m in [0.5, 1)
    y, k = 2.0 * m, e - 1             # y in [1, 2)
    j = int((y - 1.0) * 128)          # the top 7 fraction bits
    inv, t_hi, t_lo = rows[j]
    r = fma(y, inv, -1.0)
    c = fma(r, -1.0 / 6.0, 0.2)
    c = fma(r, c, -0.25)
    c = fma(r, c, 1.0 / 3.0)
    c = fma(r, c, -0.5)
    p = fma(r * r, c, r)
    hi = fma(float(k), ln2_hi, t_hi)
    lo = fma(float(k), ln2_lo, t_lo) + p
    return hi + lo


def test_exponential_method_within_two_ulp():
    tabs = _load("gen_exp_table").tables()
    rng = np.random.default_rng(11)
    xs = np.concatenate([rng.uniform(-511.0, 511.0, 600), -rng.uniform(0.0, 400.0, 400),
                         rng.uniform(-1.0, 1.0, 200), [0.0, 1.0, -1.0, 511.0, -511.0]])
    worst = max(ulps(_tang_exp(float(x), *tabs), D(float(x)).exp()) for x in xs)
    assert worst <= 2.0, worst


def test_logarithm_method_within_one_ulp():
    tabs = _load("gen_log_table").tables()
    rng = np.random.default_rng(12)
    xs = np.concatenate([np.exp(rng.uniform(np.log(2.0), 690.0, 600)), rng.uniform(50.0, 1e5, 600),
                         rng.uniform(2.0, 4.0, 200), [2.0, 4.0 - 2.0 ** -50, 1000.0, 2.0 ** 999]])
    worst = max(ulps(_table_log(float(x), *tabs), D(float(x)).ln()) for x in xs)
    assert worst <= 1.0, worst
