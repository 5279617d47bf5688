"""Why the double-FP32 residual mode stores the rows of H as three FP32 terms.

A refinement whose every residual uses the rows of H rounded to an FP32 pair
(hi + lo, 48 bits) converges to the solution of that 48-bit operator, not of
the FP64 one.  The oracle reproduces the size of that bias on the CPU:
delta_u = A^{-1} (A - A_48) u, with A_48 the operator whose H entries (the
shift c on the x diagonal, as in the library) are rounded to hi + lo.  Three
FP32 terms hold every FP64 entry exactly, so the bias vanishes.
"""

import numpy as np

from oracle import fast_solve, refined_solve, sem_1d
from oracle.sem import mode_product
from paper_2310_00226_gb300.inputs import random_rhs


def _pair(h):
    hi = h.astype(np.float32).astype(np.float64)
    return hi + (h - hi).astype(np.float32).astype(np.float64)


def _triple(h):
    hi = h.astype(np.float32).astype(np.float64)
    lo = (h - hi).astype(np.float32).astype(np.float64)
    return hi + lo + (h - hi - lo).astype(np.float32).astype(np.float64)


def _bias(u, axes, c, rnd):
    V = u.T
    out = np.zeros_like(V)
    for a, s in enumerate(axes):
        H = s.H + (c * np.eye(s.n) if a == 0 else 0.0)
        out += mode_product(V, H - rnd(H), a)
    return fast_solve(np.ascontiguousarray(out.T), *axes, c)


def test_three_fp32_terms_hold_fp64_entries_exactly():
    rng = np.random.default_rng(3)
    h = rng.standard_normal(20000) * np.exp(rng.uniform(-20, 20, 20000))
    np.testing.assert_array_equal(_triple(h), h)
    assert np.any(_pair(h) != h)


def test_48_bit_rows_bias_the_refined_solution():
    n3, k, c = (191, 63, 95), 4, 1.0
    axes = [sem_1d(k, (n + 1) // k, 0.0, 1.0) for n in n3]
    u = refined_solve(random_rhs(*n3, seed=105), *axes, c, 1)
    scale = np.abs(u).max()
    b2 = np.abs(_bias(u, axes, c, _pair)).max() / scale
    b3 = np.abs(_bias(u, axes, c, _triple)).max() / scale
    assert 1e-13 < b2 < 1e-11, b2   # measured 5.1e-13; FP64 refinement reaches ~1e-15 at this size
    assert b3 == 0.0
