"""A CPU model of the fixed-point residual's integer arithmetic, checked against
exact rational arithmetic and propagated through the solve.

The GPU kernels (paper_2310_00226_gb300/csrc/fix_kernels.cu) evaluate the
refinement residual r = f - (c + H_x (+) H_y (+) H_z) u (Eq. 12) with exact
integer products and sums.  What decides whether that is as good as FP64 is not
the size of its rounding errors but their coherence: the operator amplifies the
smooth part of a residual error by up to 1/(lambda_min + c), so a biased
rounding, or a rounding of a partial sum that varies slowly from node to node,
becomes a solution error that grows with the grid.  This model follows the
kernel's steps (balanced 28-bit chunks of U and C, three exact partial
products, the dropped low x low product, the fraction correction E round(Uh
2^-17) in an int32 sum joined to the 2^28 sum before its single rounding,
round-to-nearest conversions) with Python integers, asserts the kernel's
int64 / int32 bounds, and compares the propagated error A^-1 (r_model -
r_exact) with that of FP64 fused multiply-adds in the FP64 kernel's order, on
an operator made nearly singular (c = -0.999 lambda_min).  Planted design
mistakes -- the correction sum rounded on its own, a non-negative low chunk of
u, no fraction correction, truncating instead of rounding -- must each be
caught.  The rows of H are the oracle's (a uniform mesh: the same pattern rows
as the library's).
"""

import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import refined_solve, sem_1d
from paper_2310_00226_gb300.inputs import random_rhs

I64, I32 = 1 << 63, 1 << 31


def _bits(x):
    return int(np.float64(x).view(np.uint64))


def _to_fixed(x, s, rounding=True):
    """round(x 2^s) (halves away from zero) or trunc, from the FP64 bits."""
    b = _bits(x)
    e = (b >> 52) & 0x7FF
    m = (b & ((1 << 52) - 1)) | (1 << 52)
    sh = e - 1075 + s
    if e == 0 or sh <= -64:
        v = 0
    elif sh >= 0:
        assert sh < 10
        v = m << sh
    else:
        v = ((m + (1 << (-sh - 1))) if rounding else m) >> (-sh)
    return -v if (b >> 63) else v


def _to_f32(R, X):
    """R 2^X truncated to 24 significant bits (the kernel's FP32 conversion)."""
    if R == 0:
        return 0.0
    mag = abs(R)
    lz = 64 - mag.bit_length()
    mant = ((mag << lz) & ((1 << 64) - 1)) >> 40
    return math.copysign(mant * 2.0 ** (63 - lz + X - 23), R)


def _folded(K, q):
    return q == 0 or (K % 2 == 0 and 2 * q == K)


def _terms(K, q):
    """(dA, dB) per term: mirrored pairs for the vertex and midpoint rows."""
    if _folded(K, q):
        return [(0, None)] + [(e, -e) for e in range(1, (K if q == 0 else K // 2) + 1)]
    return [(d, None) for d in range(-q, K - q + 1)]


def _pattern_rows(n3, K, c):
    """Per local index q, the row of H (x with c on its diagonal) of an
    interior node of each axis, taken from a longer axis of the same element
    size."""
    rows = []
    for a, n in enumerate(n3):
        ne = (n + 1) // K
        big = sem_1d(K, ne + 6, 0.0, (ne + 6) / ne)
        H = np.asarray(big.H, dtype=np.float64)
        ra = []
        for q in range(K):
            i = K * ((ne + 6) // 2) + q - 1
            row = [float(H[i, i + d]) for d in range(-K, K + 1)]
            if a == 0:
                row[K] += c
            ra.append(row)
        rows.append(ra)
    return rows


def _model(n3, K, c, u, f, plant=None, with_fp64=True):
    """(r_model, r_fp64, r_exact) at every node (r_fp64 and r_exact only
    with_fp64), and the largest magnitudes of the two int64 sums and the int32
    correction sum."""
    nx, ny, nz = n3
    hq = _pattern_rows(n3, K, c)
    rsum = sum(max(sum(abs(v) for v in hq[a][q]) for q in range(K)) for a in range(3))
    t = math.floor(58.0 - math.log2(rsum))
    tab = {}
    for a in range(3):
        for q in range(K):
            for e, (dA, dB) in enumerate(_terms(K, q)):
                x = math.ldexp(hq[a][q][dA + K], t)
                C = round(x)
                E = 0 if plant == "no_fraction" else round(math.ldexp(x - C, 14))
                ch = (C + (1 << 27)) >> 28
                dc = EB = None
                if dB is not None:
                    xb = math.ldexp(hq[a][q][dB + K], t)
                    CB = round(xb)
                    dc = CB - C
                    EB = 0 if plant == "no_fraction" else round(math.ldexp(xb - CB, 14))
                tab[a, q, e] = (ch, C - (ch << 28), dc, E, EB)
    emax = lambda arr: max((_bits(v) >> 52) & 0x7FF for v in np.ravel(arr))  # noqa: E731
    s = min(1079 - emax(u), 1139 - t - emax(f))
    sF = s + t - 56
    rnd = plant != "truncate"
    U = np.vectorize(lambda v: _to_fixed(v, s, rnd), otypes=[object])(u)
    assert max(abs(v) for v in U.ravel()) <= 1 << 57
    if plant == "floor_split":
        Uh = np.vectorize(lambda v: v >> 28, otypes=[object])(U)
    else:
        Uh = np.vectorize(lambda v: (v + (1 << 27)) >> 28, otypes=[object])(U)
    Ul = U - Uh * (1 << 28)

    def get(arr, idx):
        l, j, i = idx
        return arr[idx] if (0 <= l < nz and 0 <= j < ny and 0 <= i < nx) else 0

    corr = lambda v: (v + (1 << 16)) >> 17  # noqa: E731
    r_mod, r_f64, r_ex = (np.zeros((nz, ny, nx)) for _ in range(3))
    peak = [0, 0, 0]
    for l in range(nz):
        for j in range(ny):
            for i in range(nx):
                P2 = P1 = Q = 0
                acc = float(f[l, j, i])
                ex = Fraction(acc)
                for a in range(3):
                    pos = (i, j, l)[a]
                    q = (pos + 1) % K
                    at = [lambda d: (l, j, i + d), lambda d: (l, j + d, i), lambda d: (l + d, j, i)][a]
                    for e, (dA, dB) in enumerate(_terms(K, q)):
                        ch, cl, dc, E, EB = tab[a, q, e]
                        uh, ul = get(Uh, at(dA)), get(Ul, at(dA))
                        Q += E * corr(uh)
                        if dB is not None:
                            bh, bl = get(Uh, at(dB)), get(Ul, at(dB))
                            P1 += dc * bh
                            Q += EB * corr(bh)
                            uh, ul = uh + bh, ul + bl
                            assert -I32 <= uh < I32
                        P2 += ch * uh
                        P1 += ch * ul + cl * uh
                    for d in range(-K, K + 1) if with_fp64 else ():  # FP64 FMAs (the FP64 kernel's order), exact sum
                        idx = at(d)
                        hv = hq[a][q][d + K]
                        if hv != 0.0 and all(0 <= v < m for v, m in zip(idx, (nz, ny, nx))):
                            prod = Fraction(hv) * Fraction(float(u[idx]))
                            acc = float(Fraction(acc) - prod)
                            ex -= prod
                assert abs(P2) < I64 and abs(P1) < I64 and abs(Q) < I32
                peak = [max(peak[0], abs(P2)), max(peak[1], abs(P1)), max(peak[2], abs(Q))]
                if plant == "separate_rounding":
                    T = P2 + ((P1 + (1 << 27)) >> 28) + ((Q + (1 << 24)) >> 25)
                elif plant == "truncate":
                    T = P2 + ((P1 + (Q << 3)) >> 28)
                else:
                    T = P2 + ((P1 + (Q << 3) + (1 << 27)) >> 28)
                F = _to_fixed(float(f[l, j, i]), sF, rnd)
                r_mod[l, j, i] = _to_f32(F - T, -sF)
                r_f64[l, j, i] = acc
                r_ex[l, j, i] = float(ex)
    return r_mod, r_f64, r_ex, peak


N3, K = (31, 23, 15), 4


@pytest.fixture(scope="module")
def case():
    """The operator made nearly singular (lambda_min + c = lambda_min / 1000), an
    iterate u1 near the solution, the exact residual and the propagated error of
    the FP64-FMA residual; the correct model's propagated error."""
    axes = [sem_1d(K, (n + 1) // K, 0.0, 1.0) for n in N3]
    lmin = sum(float(np.min(a.lam)) for a in axes)
    c = -0.999 * lmin
    F = random_rhs(*N3, seed=302)
    u = refined_solve(F, *axes, c, 1)
    u1 = u * (1 + 1e-11 * np.random.default_rng(1).standard_normal(u.shape))
    r_mod, r_f64, r_ex, peak = _model(N3, K, c, u1, F)
    e = lambda r: float(np.abs(refined_solve(r - r_ex, *axes, c, 1)).max() / np.abs(u).max())  # noqa: E731
    return {"axes": axes, "c": c, "F": F, "u1": u1, "r_ex": r_ex, "e": e, "peak": peak,
            "e_mod": e(r_mod), "e_f64": e(r_f64)}


def test_fixed_point_residual_is_as_accurate_as_fp64(case):
    peak = case["peak"]
    assert peak[0] < 1 << 61 and peak[1] < 1 << 62 and peak[2] < 1 << 30, [p.bit_length() for p in peak]
    # the errors of both are noise; the bound leaves room for the realisation
    assert case["e_mod"] <= 2 * case["e_f64"], (case["e_mod"], case["e_f64"])


@pytest.mark.parametrize("plant", ["separate_rounding", "floor_split", "no_fraction", "truncate"])
def test_planted_design_mistakes_are_caught(case, plant):
    r_bad, _, _, _ = _model(N3, K, case["c"], case["u1"], case["F"], plant, with_fp64=False)
    e_bad = case["e"](r_bad)
    assert e_bad > 5 * max(case["e_mod"], case["e_f64"]), (plant, e_bad, case["e_mod"], case["e_f64"])
