"""The split tiers' FP64-accurate residual in 64-bit integer fixed point.

r = f - (c + H_x (+) H_y (+) H_z) u (Eq. 12) evaluated with exact integer
products and sums on one power-of-two scale per field; its error is below one
FP64 rounding of the largest sum of |H||u| (normwise).  Checked here through
the refined solves that use it:
  * against the FP64 oracle at 1e-12 (relative L-inf), k in {1, 2, 4} (vector
    layout) and 3, 5, 6, 7, 8 (element layout), grids
    with partial 4-node chunks and short axes, both schedules that use it
    (the last sweep of "mixed", every sweep of "fp64"), BF16X3 and BF16;
  * against the same solve with FP64-FMA residuals (the two arithmetics agree
    to the refinement's floor);
  * power-of-two scaling of f scales u exactly (the scales are found on the
    device from the fields' exponents, so every integer is the same);
  * the TF32 tier's sweeps (FP64 output), against the oracle and FP64 FMAs;
  * NaN in f reaches u; plans it does not serve (k > 8, Neumann data, the
    FP32 tier) report FP64.
"""

import numpy as np
import pytest

from oracle import refined_solve, sem_1d
from paper_2310_00226_gb300.inputs import random_rhs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sem3d():
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_2310_00226_gb300 import sem3d as mod
    mod.lib()
    return mod


def _solve(sem3d, n3, k, L3, c, F, prec="bf16x3", sweeps=3, residual="mixed", exact="fixed"):
    with sem3d.Plan(*n3, k, L3, c) as p:
        p.set_precision(prec, sweeps)
        p.set_residual(residual)
        p.set_exact_residual(exact)
        kind = p.exact_residual_kind()
        f = torch.from_numpy(F).cuda()
        u = torch.full_like(f, float("nan"))
        p.solve(f, u)
        p.sync_check()
        return u.cpu().numpy(), kind


CASES = [
    ((63, 47, 95), 4, (1.0, 0.9, 1.1), 1.5),
    ((255, 127, 63), 4, (1.0, 1.0, 1.0), 2.0),
    ((29, 33, 17), 2, (1.0, 0.5, 0.25), 0.5),
    ((21, 9, 14), 1, (1.0, 1.0, 2.0), 1.0),
    ((3, 7, 11), 4, (1.0, 1.0, 1.0), 0.0),
]


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("prec,sweeps,residual", [("bf16x3", 3, "mixed"), ("bf16x3", 2, "fp64"),
                                                  ("bf16", 12, "fp64")])
def test_fixed_point_residual_matches_oracle(sem3d, case, prec, sweeps, residual):
    n3, k, L3, c = CASES[case]
    F = random_rhs(*n3, seed=300 + case)
    axes = [sem_1d(k, (n + 1) // k, 0.0, Lb) for n, Lb in zip(n3, L3)]
    ref = refined_solve(F, *axes, c, 1)
    got, kind = _solve(sem3d, n3, k, L3, c, F, prec, sweeps, residual, "fixed")
    assert kind == "fixed"
    assert np.isfinite(got).all()
    assert np.abs(got - ref).max() / np.abs(ref).max() < 1e-12, float(np.abs(got - ref).max() / np.abs(ref).max())


# k not dividing 4: the element-layout kernel (one thread per element and line)
ELEM_CASES = [((29, 17, 23), 3, (1.0, 0.8, 1.2), 1.0), ((39, 29, 19), 5, (1.0, 1.0, 1.0), 0.5),
              ((47, 35, 23), 6, (1.0, 1.0, 1.0), 2.0), ((27, 41, 13), 7, (1.0, 1.5, 0.5), 1.0),
              ((63, 31, 47), 8, (1.0, 1.0, 1.0), 0.0)]


@pytest.mark.parametrize("case", range(len(ELEM_CASES)))
@pytest.mark.parametrize("sweeps,residual", [(3, "mixed"), (2, "fp64")])
def test_fixed_point_residual_element_layout(sem3d, case, sweeps, residual):
    n3, k, L3, c = ELEM_CASES[case]
    F = random_rhs(*n3, seed=340 + case)
    axes = [sem_1d(k, (n + 1) // k, 0.0, Lb) for n, Lb in zip(n3, L3)]
    ref = refined_solve(F, *axes, c, 1)
    got, kind = _solve(sem3d, n3, k, L3, c, F, "bf16x3", sweeps, residual, "fixed")
    assert kind == "fixed"
    assert np.isfinite(got).all()
    assert np.abs(got - ref).max() / np.abs(ref).max() < 1e-12, float(np.abs(got - ref).max() / np.abs(ref).max())
    fp, _ = _solve(sem3d, n3, k, L3, c, F, "bf16x3", sweeps, residual, "fp64")
    assert np.abs(got - fp).max() / np.abs(fp).max() < 1e-13


@pytest.mark.parametrize("n3,k", [((63, 47, 95), 4), ((29, 17, 23), 3)])
def test_tf32_tier_with_fixed_point_residuals(sem3d, n3, k):
    # the TF32 tier's sweeps read r in FP64 (the kernels' FP64 output mode)
    L3, c = (1.0, 0.9, 1.1), 1.5
    F = random_rhs(*n3, seed=350 + k)
    axes = [sem_1d(k, (n + 1) // k, 0.0, Lb) for n, Lb in zip(n3, L3)]
    ref = refined_solve(F, *axes, c, 1)
    got, kind = _solve(sem3d, n3, k, L3, c, F, "tf32", 6, "mixed", "fixed")
    assert kind == "fixed"
    assert np.abs(got - ref).max() / np.abs(ref).max() < 1e-12, float(np.abs(got - ref).max() / np.abs(ref).max())
    fp, kind = _solve(sem3d, n3, k, L3, c, F, "tf32", 6, "mixed", "fp64")
    assert kind == "fp64"
    assert np.abs(got - fp).max() / np.abs(fp).max() < 1e-13


@pytest.mark.parametrize("case", [0, 1, 2])
def test_fixed_point_and_fp64_residuals_agree(sem3d, case):
    n3, k, L3, c = CASES[case]
    F = random_rhs(*n3, seed=320 + case)
    fx, kind_fx = _solve(sem3d, n3, k, L3, c, F, exact="fixed")
    fp, kind_fp = _solve(sem3d, n3, k, L3, c, F, exact="fp64")
    assert (kind_fx, kind_fp) == ("fixed", "fp64")
    assert np.abs(fx - fp).max() / np.abs(fp).max() < 1e-13


def test_no_coherent_bias_under_strong_amplification(sem3d):
    # With c close to -lambda_min the operator amplifies the smooth part of a
    # residual error by ~1/(lambda_min + c): a biased rounding in the fixed-
    # point residual (or a row-sum error of the fixed-point rows) would show
    # here as a difference from the FP64-residual solve far above the FP64
    # residual's own noise.
    n3, k, L3 = (63, 47, 95), 4, (1.0, 0.9, 1.1)
    lmin = sum(float(np.min(sem_1d(k, (n + 1) // k, 0.0, Lb).lam)) for n, Lb in zip(n3, L3))
    c = -0.99 * lmin
    F = random_rhs(*n3, seed=333)
    fx, _ = _solve(sem3d, n3, k, L3, c, F, sweeps=3)
    fp, _ = _solve(sem3d, n3, k, L3, c, F, sweeps=3, exact="fp64")
    assert np.isfinite(fx).all() and np.isfinite(fp).all()
    assert np.abs(fx - fp).max() / np.abs(fp).max() < 1e-13, float(np.abs(fx - fp).max() / np.abs(fp).max())


@pytest.mark.parametrize("e", [40, -40])
def test_power_of_two_scaling_is_exact(sem3d, e):
    n3, k, L3, c = CASES[0]
    F = random_rhs(*n3, seed=330)
    base, _ = _solve(sem3d, n3, k, L3, c, F, sweeps=2, residual="fp64")
    scaled, _ = _solve(sem3d, n3, k, L3, c, np.ldexp(F, e), sweeps=2, residual="fp64")
    assert np.array_equal(scaled, np.ldexp(base, e))


def test_wide_dynamic_range_matches_oracle(sem3d):
    # f spanning 12 decades (one global scale: small entries get the field's
    # absolute resolution; the normwise result is still FP64-accurate)
    n3, k, L3, c = (63, 31, 47), 4, (1.0, 1.0, 1.0), 1.0
    rng = np.random.default_rng(7)
    F = random_rhs(*n3, seed=331) * np.exp(rng.uniform(-14, 14, size=n3[::-1]))
    axes = [sem_1d(k, (n + 1) // k, 0.0, Lb) for n, Lb in zip(n3, L3)]
    ref = refined_solve(F, *axes, c, 1)
    got, _ = _solve(sem3d, n3, k, L3, c, F)
    assert np.abs(got - ref).max() / np.abs(ref).max() < 1e-12


def test_nan_in_f_reaches_u(sem3d):
    n3, k, L3, c = (31, 15, 23), 4, (1.0, 1.0, 1.0), 1.0
    F = random_rhs(*n3, seed=332)
    F[5, 3, 7] = np.nan
    got, _ = _solve(sem3d, n3, k, L3, c, F, sweeps=2, residual="fp64")
    assert np.isnan(got).any()


def test_kind_reporting(sem3d):
    with sem3d.Plan(31, 31, 31, 4, (1.0, 1.0, 1.0), 1.0) as p:
        assert p.exact_residual_kind() == "fp64"  # FP64 tier
        p.set_precision("bf16x3", 3)
        assert p.exact_residual_kind() == "fixed"
        p.set_exact_residual("fp64")
        assert p.exact_residual_kind() == "fp64"
        p.set_precision("tf32", 3)
        p.set_exact_residual("fixed")
        assert p.exact_residual_kind() == "fixed"  # TF32 tier: every sweep
        p.set_precision("fp32", 2)
        assert p.exact_residual_kind() == "fp64"  # FP32 tier: FP64 residuals
    with sem3d.Plan(29, 29, 29, 3, (1.0, 1.0, 1.0), 1.0) as p:
        p.set_precision("bf16x3", 3)
        assert p.exact_residual_kind() == "fixed"  # k = 3: the element-layout kernel
    with sem3d.Plan(35, 35, 35, 9, (1.0, 1.0, 1.0), 1.0) as p:
        p.set_precision("bf16x3", 3)
        assert p.exact_residual_kind() == "fp64"  # k > 8
    with sem3d.Plan(33, 33, 33, 4, (1.0, 1.0, 1.0), 1.0, bc="neumann") as p:
        p.set_precision("bf16x3", 3)
        assert p.exact_residual_kind() == "fp64"  # Neumann rows
    with sem3d.Plan(7, 7, 7, 2) as p:
        assert sem3d.lib().sem3d_set_exact_residual(p._h, 7) != 0  # unknown kind
