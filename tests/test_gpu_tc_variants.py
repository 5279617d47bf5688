"""The two tensor-core kernels of the split tiers and the autotuner that picks one.

Variant 0 runs one CTA per 128 x 256 output tile (W multicast across clusters
of 4 CTAs); variant 1 runs one cta_group::2 MMA per pair of SMs on 256 x 256
tiles.  Both issue the same MMAs in the same K order into FP32 accumulators, so
every pass, and therefore every solve, must be bit-identical between them; the
tests pin each variant through the C ABI and compare whole fields, on ragged
grids that leave partial M, N and K tiles, in every epilogue mode the solve
uses (split output, division, FP64 store / accumulate, the double-FP32 modes
of the mixed and double-FP32 residual schemes) and in the one-product BF16
tier.  Refined results are also held to the oracle (1e-12).
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


def _solve(sem3d, n3, k, L3, c, prec, sweeps, residual, variant, F):
    with sem3d.Plan(*n3, k, L3, c) as p:
        for ax in range(3):
            p.set_tc_config(ax, variant)
        p.set_precision(prec, sweeps)
        p.set_residual(residual)
        for ax in range(3):
            assert p.tc_config(ax) == variant  # a pinned shape is not re-measured
        f = torch.from_numpy(F).cuda()
        u = torch.full_like(f, float("nan"))
        p.solve(f, u)
        p.sync_check()
        return u.cpu().numpy()


CASES = [
    ((63, 47, 95), 4, (1.0, 0.9, 1.1), 1.5),
    ((255, 127, 63), 4, (1.0, 1.0, 1.0), 2.0),
    ((129, 257, 65), 2, (1.0, 0.5, 0.25), 0.5),
    ((383, 63, 95), 4, (1.0, 1.0, 1.0), 1.0),
]
TIERS = [("bf16x3", 0, "mixed"), ("bf16x3", 3, "mixed"), ("bf16x3", 3, "fp64"), ("bf16x3", 2, "df"),
         ("bf16", 0, "mixed")]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_pair_kernel_is_bit_identical_to_single_cta_kernel(sem3d, case):
    n3, k, L3, c = CASES[case]
    F = random_rhs(*n3, seed=40 + case)
    sx, sy, sz = (sem_1d(k, (n + 1) // k, 0.0, Lb) for n, Lb in zip(n3, L3))
    ref = refined_solve(F, sx, sy, sz, c, 1)
    for prec, sweeps, residual in TIERS:
        single = _solve(sem3d, n3, k, L3, c, prec, sweeps, residual, 0, F)
        pair = _solve(sem3d, n3, k, L3, c, prec, sweeps, residual, 1, F)
        assert np.isfinite(pair).all()
        assert np.array_equal(pair, single), (prec, sweeps, residual, float(np.abs(pair - single).max()))
        if prec == "bf16x3" and sweeps == 3:
            assert np.abs(pair - ref).max() / np.abs(ref).max() < 1e-12


def test_autotuner_records_a_choice_per_axis(sem3d):
    # An unseen shape: set_precision measures both kernels per pass and records
    # 0 or 1; the solve then matches the oracle whichever was chosen.
    n3, k, L3, c = (191, 95, 127), 4, (1.0, 1.0, 1.0), 1.0
    F = random_rhs(*n3, seed=7)
    sx, sy, sz = (sem_1d(k, (n + 1) // k, 0.0, Lb) for n, Lb in zip(n3, L3))
    ref = refined_solve(F, sx, sy, sz, c, 1)
    with sem3d.Plan(*n3, k, L3, c) as p:
        p.set_precision("bf16x3", 3)
        choice = [p.tc_config(ax) for ax in range(3)]
        assert all(v in (0, 1) for v in choice)
        f = torch.from_numpy(F).cuda()
        u = torch.empty_like(f)
        p.solve(f, u)
        p.sync_check()
        assert np.abs(u.cpu().numpy() - ref).max() / np.abs(ref).max() < 1e-12
        p.set_tc_config(1, 1 - choice[1])   # a pin replaces the measured choice
        assert p.tc_config(1) == 1 - choice[1]


def test_set_tc_config_validates(sem3d):
    with sem3d.Plan(31, 31, 31, 2, (1.0, 1.0, 1.0), 0.0) as p:
        with pytest.raises(sem3d.Sem3dError):
            p.set_tc_config(3, 0)
        with pytest.raises(sem3d.Sem3dError):
            p.set_tc_config(0, 2)


TF32_CASES = [((63, 47, 95), 4, (1.0, 0.9, 1.1), 1.5), ((287, 257, 259), 2, (1.0, 1.0, 1.0), 1.0)]


@pytest.mark.parametrize("case", range(len(TF32_CASES)))
def test_tf32_pair_kernel_is_bit_identical_to_single_cta_kernel(sem3d, case):
    # The TF32 tier's two kernels (kind::tf32; one CTA per tile with W
    # multicast, or a cta_group::2 pair) on ragged grids, bare and refined.
    n3, k, L3, c = TF32_CASES[case]
    F = random_rhs(*n3, seed=60 + case)
    for sweeps in (0, 3):
        single = _solve(sem3d, n3, k, L3, c, "tf32", sweeps, "mixed", 0, F)
        pair = _solve(sem3d, n3, k, L3, c, "tf32", sweeps, "mixed", 1, F)
        assert np.isfinite(pair).all()
        assert np.array_equal(pair, single), (sweeps, float(np.abs(pair - single).max()))


def test_tf32_autotuner_records_a_choice_per_axis(sem3d):
    n3, k = (191, 95, 127), 4
    with sem3d.Plan(*n3, k, (1.0, 1.0, 1.0), 1.0) as p:
        p.set_precision("tf32", 0)
        assert all(p.tc_config(ax) in (0, 1) for ax in range(3))
