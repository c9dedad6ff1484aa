"""FP64 oracle: sixth-order compact staggered interpolation and first derivative (Sec. 3.1).

TEST INFRASTRUCTURE (see oracle/gas.py header). Not used by the product path.

The paper discretises space with fourth- or sixth-order compact finite differences (Lele 1992) on
a staggered grid (Fig. 1) and leaves the operator details to a thesis that is not available. The
reading used here (the CUDA path implements the same operator, independently):

Along one grid line with n cells, "centre" nodes sit at positions k + 1/2 (k = 0..n-1) and "face"
nodes at positions i (i = 0..n), in index units (spacing 1).

* Interior rows, midpoint interpolation:   alpha (g_{i-1} + g_{i+1}) + g_i
      = a/2 (f_{i+1/2} + f_{i-1/2}) + b/2 (f_{i+3/2} + f_{i-3/2}),   alpha = 3/10, a = 3/2, b = 1/10
* Interior rows, staggered first derivative: alpha (g'_{i-1} + g'_{i+1}) + g'_i
      = a (f_{i+1/2} - f_{i-1/2}) + b/3 (f_{i+3/2} - f_{i-3/2}),       alpha = 9/62, a = 63/62, b = 17/62
* Rows whose interior stencil would leave the line are explicit (identity on the left-hand side):
  the value or derivative at the output position of the Lagrange polynomial through the five
  input nodes nearest that end of the line. With a known wall value at position 0 ("wall" variant,
  centre -> face only), the five nodes are the wall value and the first four centres.

Each operator is the linear map y = A^{-1} (B x) with A tridiagonal; the oracle forms A and B
explicitly and calls a banded solver and a sparse product.
"""
from __future__ import annotations

from fractions import Fraction
from functools import lru_cache

import numpy as np
import scipy.linalg
import scipy.sparse

INTERP6 = dict(alpha=Fraction(3, 10), a=Fraction(3, 2), b=Fraction(1, 10))
DERIV6 = dict(alpha=Fraction(9, 62), a=Fraction(63, 62), b=Fraction(17, 62))
CLOSURE_POINTS = 5


def lagrange_weights(nodes, x, derivative):
    """Exact weights w_k with p(x) = sum_k w_k f_k (or p'(x)) for the interpolating polynomial."""
    nodes = [Fraction(v) for v in nodes]
    x = Fraction(x)
    w = []
    for k, xk in enumerate(nodes):
        others = [xm for m, xm in enumerate(nodes) if m != k]
        den = Fraction(1)
        for xm in others:
            den *= (xk - xm)
        if not derivative:
            num = Fraction(1)
            for xm in others:
                num *= (x - xm)
        else:
            num = Fraction(0)
            for skip in range(len(others)):
                term = Fraction(1)
                for m, xm in enumerate(others):
                    if m != skip:
                        term *= (x - xm)
                num += term
        w.append(num / den)
    return w


@lru_cache(maxsize=None)
def operator_matrices(kind, direction, n, wall):
    """Return (A as dense banded (3, m) for solve_banded, B as csr (m, n_in_aug)).

    kind: 'I' (interpolation) or 'D' (first derivative); direction: 'cf' (centre -> face,
    n inputs, n + 1 outputs) or 'fc' (face -> centre, n + 1 inputs, n outputs); wall: if True
    (cf only) the input vector is augmented with the wall value as its first entry.
    """
    coef = INTERP6 if kind == 'I' else DERIV6
    deriv = kind == 'D'
    if direction == 'cf':
        m, n_in = n + 1, n
        in_pos = [Fraction(2 * k + 1, 2) for k in range(n)]
        out_pos = [Fraction(i) for i in range(n + 1)]
        interior = range(2, n - 1)
    else:
        m, n_in = n, n + 1
        in_pos = [Fraction(i) for i in range(n + 1)]
        out_pos = [Fraction(2 * k + 1, 2) for k in range(n)]
        interior = range(1, n - 1)
    off = 1 if wall else 0
    if wall:
        assert direction == 'cf'
        in_pos = [Fraction(0)] + in_pos
    A = np.zeros((3, m))
    A[1, :] = 1.0
    rows, cols, vals = [], [], []

    def put(r, c, v):
        rows.append(r)
        cols.append(c)
        vals.append(float(v))

    interior = set(interior)
    for r in range(m):
        x = out_pos[r]
        if r in interior:
            alpha = coef['alpha']
            if r - 1 >= 0:
                A[2, r - 1] = float(alpha)      # sub-diagonal entry of row r
            if r + 1 < m:
                A[0, r + 1] = float(alpha)      # super-diagonal entry of row r
            # input nodes at x -/+ 1/2 and x -/+ 3/2
            idx = {}
            for k, p in enumerate(in_pos):
                d = p - x
                if d in (Fraction(-3, 2), Fraction(-1, 2), Fraction(1, 2), Fraction(3, 2)):
                    idx[d] = k
            a, b = coef['a'], coef['b']
            if deriv:
                put(r, idx[Fraction(1, 2)], a)
                put(r, idx[Fraction(-1, 2)], -a)
                put(r, idx[Fraction(3, 2)], b / 3)
                put(r, idx[Fraction(-3, 2)], -b / 3)
            else:
                put(r, idx[Fraction(1, 2)], a / 2)
                put(r, idx[Fraction(-1, 2)], a / 2)
                put(r, idx[Fraction(3, 2)], b / 2)
                put(r, idx[Fraction(-3, 2)], b / 2)
        else:
            left = x < Fraction(len(out_pos), 2)
            if left:
                ks = list(range(0, CLOSURE_POINTS))
            else:
                ks = list(range(len(in_pos) - CLOSURE_POINTS, len(in_pos)))
            w = lagrange_weights([in_pos[k] for k in ks], x, deriv)
            for k, wk in zip(ks, w):
                if wk != 0:
                    put(r, k, wk)
    B = scipy.sparse.csr_matrix((vals, (rows, cols)), shape=(m, n_in + off))
    return A, B


def apply(f, axis, kind, direction, wall_value=None):
    """Apply the operator along ``axis`` of array f (index-space result, spacing 1)."""
    f = np.asarray(f, dtype=np.float64)
    fm = np.moveaxis(f, axis, 0)
    shape = fm.shape
    n_in = shape[0]
    n = n_in if direction == 'cf' else n_in - 1
    wall = wall_value is not None
    A, B = operator_matrices(kind, direction, n, wall)
    x = fm.reshape(n_in, -1)
    if wall:
        wv = np.broadcast_to(np.asarray(wall_value, dtype=np.float64).reshape(1, -1), (1, x.shape[1]))
        x = np.vstack([wv, x])
    rhs = B @ x
    y = scipy.linalg.solve_banded((1, 1), A, rhs)
    out = y.reshape((A.shape[1],) + shape[1:])
    return np.moveaxis(out, 0, axis)


def icf(f, axis, wall_value=None):
    return apply(f, axis, 'I', 'cf', wall_value)


def dcf(f, axis, wall_value=None):
    return apply(f, axis, 'D', 'cf', wall_value)


def ifc(f, axis):
    return apply(f, axis, 'I', 'fc')


def dfc(f, axis):
    return apply(f, axis, 'D', 'fc')


# ---------------------------------------------------------------------------------------------
# Periodic lines (the spanwise direction of three-dimensional cases)
# ---------------------------------------------------------------------------------------------
# A periodic line of n cells has centres at k + 1/2 and faces at i (i = 0..n-1; face n is face 0).
# Every row is an interior row of the sixth-order schemes above, with indices taken modulo n; A is
# then circulant and the oracle solves it densely.

@lru_cache(maxsize=None)
def periodic_matrices(kind, direction, n):
    """Dense (A, B), both (n, n), of the periodic operator; kind 'I' or 'D', direction 'cf'
    (centres -> faces) or 'fc' (faces -> centres)."""
    coef = INTERP6 if kind == 'I' else DERIV6
    a, b, alpha = float(coef['a']), float(coef['b']), float(coef['alpha'])
    A = np.zeros((n, n))
    B = np.zeros((n, n))
    for r in range(n):
        A[r, r] = 1.0
        A[r, (r - 1) % n] += alpha
        A[r, (r + 1) % n] += alpha
        # inputs at offsets -3/2, -1/2, +1/2, +3/2 from output r
        if direction == 'cf':          # face r; centre k sits at k + 1/2
            km3, km1, kp1, kp3 = r - 2, r - 1, r, r + 1
        else:                          # centre r + 1/2; face i sits at i
            km3, km1, kp1, kp3 = r - 1, r, r + 1, r + 2
        if kind == 'I':
            w = {km3: b / 2, km1: a / 2, kp1: a / 2, kp3: b / 2}
        else:
            w = {km3: -b / 3, km1: -a, kp1: a, kp3: b / 3}
        for k, v in w.items():
            B[r, k % n] += v
    return A, B


def apply_periodic(f, axis, kind, direction):
    """Apply the periodic operator along ``axis`` (index-space result, spacing 1)."""
    f = np.asarray(f, dtype=np.float64)
    fm = np.moveaxis(f, axis, 0)
    n = fm.shape[0]
    A, B = periodic_matrices(kind, direction, n)
    x = fm.reshape(n, -1)
    y = np.linalg.solve(A, B @ x)
    return np.moveaxis(y.reshape(fm.shape), 0, axis)


def icf_p(f, axis):
    return apply_periodic(f, axis, 'I', 'cf')


def ifc_p(f, axis):
    return apply_periodic(f, axis, 'I', 'fc')


def dcf_p(f, axis):
    return apply_periodic(f, axis, 'D', 'cf')


def dfc_p(f, axis):
    return apply_periodic(f, axis, 'D', 'fc')
