"""The binary64 exponential, quotient, reciprocal and logarithm of the FP64 closure
(hyp_fp64_fast): within 2 ulp of the exact result over the closure's argument ranges (the exact
result from numpy's long double arithmetic, at least 64 significand bits), and equal to CUDA's own
functions where the arguments leave the fast ranges."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _ulp_error(got, exact):
    """|got - exact| in units of the last place of the binary64 nearest to exact."""
    ref = exact.astype(np.float64)
    ulp = np.spacing(np.abs(ref))
    return (np.abs(got.astype(np.longdouble) - exact) / ulp.astype(np.longdouble)).astype(np.float64)


def _run(fn, a=None, b=None):
    import torch
    from paper_2210_05547_gb300 import abi as A
    n = (a if a is not None else b).size
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    A.fp64_fast(fn, out, a=None if a is None else torch.as_tensor(a).cuda(),
                b=None if b is None else torch.as_tensor(b).cuda())
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_exp_within_two_ulp():
    rng = np.random.default_rng(7)
    x = np.concatenate([
        rng.uniform(-511.9, 511.9, 400_000),               # the whole fast range
        -rng.uniform(0.0, 400.0, 200_000),                  # -T_a/T, -theta/T of the closure
        rng.uniform(-1.0, 1.0, 200_000),                    # near zero
        rng.uniform(-1e-6, 1e-6, 50_000),
        np.array([0.0, -0.0, 1.0, -1.0, np.log(2.0), 511.0, -511.0]),
    ])
    got = _run(0, a=x)
    exact = np.exp(x.astype(np.longdouble))
    err = _ulp_error(got, exact)
    assert err.max() <= 2.0, (err.max(), x[np.argmax(err)])


def test_exp_outside_the_fast_range_is_cudas():
    import torch
    x = np.array([512.0, 700.0, 709.5, 720.0, -600.0, -745.0, -800.0, np.inf, -np.inf, np.nan])
    got = _run(0, a=x)
    want = torch.exp(torch.as_tensor(x).cuda()).cpu().numpy()
    assert np.array_equal(got, want, equal_nan=True)


def test_quotient_and_reciprocal_within_two_ulp():
    rng = np.random.default_rng(8)
    n = 400_000
    a = rng.uniform(-1.0, 1.0, n) * np.exp(rng.uniform(-80.0, 80.0, n))
    b = rng.choice([-1.0, 1.0], n) * np.exp(rng.uniform(-80.0, 80.0, n))
    q = _run(1, a=a, b=b)
    r = _run(2, b=b)
    eq = _ulp_error(q, a.astype(np.longdouble) / b.astype(np.longdouble))
    er = _ulp_error(r, 1.0 / b.astype(np.longdouble))
    assert eq.max() <= 2.0, (eq.max(), a[np.argmax(eq)], b[np.argmax(eq)])
    assert er.max() <= 2.0, (er.max(), b[np.argmax(er)])


def test_quotient_outside_the_fast_range_is_cudas():
    import torch
    b = np.array([1e-200, -1e-300, 1e200, 0.0, -0.0, np.inf, np.nan, 2.0 ** -121, 2.0 ** 121])
    a = np.full(b.size, 3.0)
    got = _run(1, a=a, b=b)
    want = (torch.as_tensor(a).cuda() / torch.as_tensor(b).cuda()).cpu().numpy()
    assert np.array_equal(got, want, equal_nan=True)
    got_r = _run(2, b=b)
    want_r = (1.0 / torch.as_tensor(b).cuda()).cpu().numpy()
    assert np.array_equal(got_r, want_r, equal_nan=True)


def test_log_within_two_ulp():
    rng = np.random.default_rng(9)
    x = np.concatenate([
        np.exp(rng.uniform(np.log(2.0), 690.0, 300_000)),   # the whole fast range
        rng.uniform(50.0, 1.0e5, 300_000),                  # temperatures of the closure
        rng.uniform(2.0, 4.0, 100_000),                     # the first binade
        np.array([2.0, 2.0 + 2.0 ** -51, 4.0 - 2.0 ** -50, 1024.0, 1000.0, 2.0 ** 999]),
    ])
    got = _run(3, a=x)
    err = _ulp_error(got, np.log(x.astype(np.longdouble)))
    assert err.max() <= 2.0, (err.max(), x[np.argmax(err)])


def test_log_outside_the_fast_range_is_cudas():
    import torch
    x = np.array([1.999, 1.0, 0.5, 1e-300, 0.0, -1.0, 2.0 ** 1000, 1e308, np.inf, np.nan])
    got = _run(3, a=x)
    want = torch.log(torch.as_tensor(x).cuda()).cpu().numpy()
    assert np.array_equal(got, want, equal_nan=True)
