"""Why the mixed path's line operators are compensated where they are, checked with the oracle on
the CPU (reading 22 of the design): the compact operators of the right-hand side (Sec. 3.1) are
replaced by binary32 solves in two ways and the right-hand side is compared with the FP64 one.

* As the mixed kernels do: derivatives solve A y = B f with B f formed in binary64 (the
  differences where the cancellation happens) and the tridiagonal solve in binary32;
  interpolations solve for their correction to the two-point average (B f - A avg in binary64,
  the solve in binary32), a stand-in for their double-word recurrence, which is closer still.
  The right-hand side stays within 1e-6 of max|R| per field.
* With the inputs themselves rounded to binary32 (plain binary32 operators), some field misses
  that bound several times over (9e-6 here, 2e-5 to 1e-4 on the 2048 x 256 case): the rounding of
  a field value is then carried into its derivative.
"""
import numpy as np
import pytest
import scipy.linalg

from gpu_util import oracle_case
from oracle import compact as C
from oracle import flow as F
from paper_2210_05547_gb300 import inputs as I


def _solve32(A, rhs):
    return scipy.linalg.solve_banded((1, 1), A.astype(np.float32),
                                     rhs.astype(np.float32)).astype(np.float64)


def _apply_factory(kind_of_split):
    def apply(f, axis, kind, direction, wall_value=None):
        f = np.asarray(f, dtype=np.float64)
        fm = np.moveaxis(f, axis, 0)
        shape = fm.shape
        n_in = shape[0]
        n = n_in if direction == "cf" else n_in - 1
        wall = wall_value is not None
        A, B = C.operator_matrices(kind, direction, n, wall)
        x = fm.reshape(n_in, -1)
        if wall:
            wv = np.broadcast_to(np.asarray(wall_value, dtype=np.float64).reshape(1, -1),
                                 (1, x.shape[1]))
            x = np.vstack([wv, x])
        if kind_of_split == "plain":
            y = _solve32(A, B @ x.astype(np.float32).astype(np.float64))
        elif kind == "D":
            y = _solve32(A, B @ x)
        else:
            exact = scipy.linalg.solve_banded((1, 1), A, B @ x)
            xs = x[1:] if wall else x
            avg = exact.copy()
            if direction == "cf" and xs.shape[0] == exact.shape[0] - 1:
                avg[1:-1] = 0.5 * (xs[:-1] + xs[1:])
            elif direction == "fc":
                avg[:] = 0.5 * (xs[:-1] + xs[1:])
            a_avg = A[1][:, None] * avg
            a_avg[:-1] += A[0][1:, None] * avg[1:]
            a_avg[1:] += A[2][:-1, None] * avg[:-1]
            y = avg + _solve32(A, B @ x - a_avg)
        out = y.reshape((A.shape[1],) + shape[1:])
        return np.moveaxis(out, 0, axis)
    return apply


def _errors(table, cfg, monkeypatch, split):
    case = oracle_case(table, cfg)
    ref = F.unpack(5, cfg["nx"], cfg["ny"], F.rhs(case, case.U0))
    with monkeypatch.context() as m:
        m.setattr(C, "apply", _apply_factory(split))
        got = F.unpack(5, cfg["nx"], cfg["ny"], F.rhs(case, case.U0))
    return {k: float(np.abs(got[k] - ref[k]).max() / np.abs(ref[k]).max()) for k in ref}


@pytest.mark.parametrize("cfg", [I.sbli_case(128, 48, seed=3), I.sbli_case(192, 64, seed=4)],
                         ids=["sbli_128x48", "sbli_192x64"])
def test_compensated_binary32_operators_within_1e6(table, cfg, monkeypatch):
    err = _errors(table, cfg, monkeypatch, "compensated")
    assert max(err.values()) < 1e-6, err
    assert max(err.values()) > 1e-9, err           # the binary32 solves are really in the result


def test_plain_binary32_operators_miss_the_bound(table, monkeypatch):
    err = _errors(table, I.sbli_case(128, 48, seed=3), monkeypatch, "plain")
    assert max(err.values()) > 5e-6, err
