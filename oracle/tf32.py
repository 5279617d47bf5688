"""TF32 rounding and the fast solve with rounded operands.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Section 3.7 (the comparison with a JAX implementation, Table 10) runs the
single-precision solve twice on the same GPU: once with the TF32 format, which
the tensor cores read for FP32 matrix products unless it is switched off, and
once in plain FP32.  TF32 keeps FP32's 8-bit exponent but only a 10-bit
mantissa (11 significant bits), so every operand of a mode product is rounded
to about 3.3 decimal digits, while products are summed in FP32.  Table 10 shows
the consequence for the Q^5 method: the l2 error stops at ~1e-3 once the grid
reaches 79^3, where plain FP32 reaches ~1e-6.

``tf32_round`` states that rounding from its definition (round to the nearest
number with 11 significant bits, ties to even, with FP32's exponent range and
subnormal spacing); ``fast_solve_rounded`` is Eq. 13 with a rounding applied to
every operand of the six mode products.
"""

from __future__ import annotations

import numpy as np

from .sem import Sem1D, mode_product


def tf32_round(x) -> np.ndarray:
    """Round FP32 values (anything else is first converted to FP32) to the
    nearest TF32 number, ties to even; returns FP32 values.

    A finite nonzero x is m * 2^e with 0.5 <= |m| < 1, so its leading bit is
    2^(e-1) and 11 significant bits end at the quantum 2^(e-11).  Below FP32's
    smallest normal 2^-126 (e <= -126) the spacing stays that of the binade
    [2^-126, 2^-125), i.e. 2^-136: the exponent is clamped at -125.  Results
    beyond FP32's range become infinities; zeros, infinities and NaN pass.
    """
    with np.errstate(over="ignore"):
        x32 = np.asarray(x, dtype=np.float32)
    x64 = x32.astype(np.float64)
    _, e = np.frexp(x64)
    e = np.maximum(e, -125)
    with np.errstate(over="ignore", invalid="ignore"):
        q = np.round(np.ldexp(x64, 11 - e))  # numpy rounds halves to even
        r = np.ldexp(q, e - 11).astype(np.float32)
    return np.where(np.isfinite(x32), r, x32)


def tf32_operand(a) -> np.ndarray:
    """FP64 array -> FP32 -> TF32, returned as FP64 (the operand a TF32 mode
    product reads)."""
    with np.errstate(over="ignore"):
        a32 = np.asarray(a, dtype=np.float64).astype(np.float32)
    return tf32_round(a32).astype(np.float64)


def fast_solve_rounded(F: np.ndarray, sx: Sem1D, sy: Sem1D, sz: Sem1D, c: float, rnd=tf32_operand) -> np.ndarray:
    """Eq. 13 with every operand of the six mode products passed through
    ``rnd``: the right-hand side, the six matrices T^{-1} and T, and the
    outputs of the first five products (the third after the division by
    lambda_x + lambda_y + lambda_z + c).  Products are summed in FP64; the last
    product's output is returned unrounded.

    Order: x, y, z with T^{-1}, then x, y, z with T (the order of the TF32
    tier, whose passes each contract the fastest axis of their input).  The
    paper's forward order is z, y, x; mode products along different axes
    commute, so with ``rnd`` the identity this equals ``fast_solve`` up to
    FP64 rounding (pinned).  F and the result are (nz, ny, nx) arrays.
    """
    s = (sx, sy, sz)
    U = rnd(np.asarray(F, dtype=np.float64).T)  # the paper's U(i, j, l)
    for axis in (0, 1, 2):
        U = mode_product(U, rnd(s[axis].Tinv), axis)
        if axis == 2:
            U = U / (sx.lam[:, None, None] + sy.lam[None, :, None] + sz.lam[None, None, :] + c)
        U = rnd(U)
    for axis in (0, 1, 2):
        U = mode_product(U, rnd(s[axis].T), axis)
        if axis < 2:
            U = rnd(U)
    return np.ascontiguousarray(U.T)
