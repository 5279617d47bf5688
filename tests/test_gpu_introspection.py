"""Introspection entry points on the GPU: sem3d_get_eigs against the oracle's
eigendecomposition (Section 2.3), and the launch accounting that bench.py's
`gpu_launches` and per-kernel timings rely on (sem3d_launch_count,
sem3d_profile / sem3d_profile_read), checked against the structure of each
tier's solve.

Expected launches of one solve with s FP64 refinement sweeps on a grid whose
x pitch is padded (Px > nx), k = 2:
  FP64   : 6 DMMA passes per solve, one FP64 residual per sweep     6(s+1) + s
  FP32   : 6 FFMA passes per solve, one FP64 residual per sweep     6(s+1) + s
  TF32   : conversion + 6 passes per solve, one residual per sweep  7(s+1) + s
  BF16x3 : one split, 6 passes per solve; s-1 double-FP32 residuals
           (one launch each) and one FP64 residual with a split output
           (stencil + pad zeroing: two launches)                    1 + 6(s+1) + (s-1) + 2
"""

import numpy as np
import pytest

from oracle import sem_1d
from paper_2310_00226_gb300.inputs import random_rhs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N3, K, L3, C = (63, 39, 47), 2, (1.0, 0.7, 1.3), 2.0


@pytest.fixture(scope="module")
def sem3d():
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_2310_00226_gb300 import sem3d as mod
    mod.lib()
    return mod


def test_get_eigs_matches_oracle(sem3d):
    with sem3d.Plan(*N3, K, L3, C) as p:
        for a in range(3):
            s = sem_1d(K, (N3[a] + 1) // K, 0.0, L3[a])
            lam, T = p.eigs(a, with_vectors=True)
            np.testing.assert_allclose(lam, s.lam, rtol=1e-12)
            assert np.all(np.diff(lam) > 0)
            # same eigenvectors up to the sign of each column (a column's largest-magnitude
            # entry is made positive on both sides, but antisymmetric modes have two of opposite sign)
            sgn = np.sign(np.sum(T * s.T, axis=0))
            assert np.all(sgn != 0)
            assert np.abs(T * sgn[None, :] - s.T).max() <= 1e-10 * np.abs(s.T).max()
            # and they diagonalise H = M^{-1} S: H T = T diag(lambda)
            HT = s.H @ T
            assert np.abs(HT - T * lam[None, :]).max() <= 1e-10 * np.abs(HT).max()


@pytest.mark.parametrize("tier,sweeps,expected", [
    ("fp64", 1, 6 * 2 + 1),
    ("fp32", 2, 6 * 3 + 2),
    # TF32: 4 solves of 7 launches; fixed-point residuals (f's and u's exponents, conversion, stencil; then
    # u's exponent, conversion, stencil)
    ("tf32", 3, 7 * 4 + 4 + 3 + 3),
    # split (which also takes f's exponent), 4 solves, 2 double-FP32 residuals, the
    # fixed-point residual (u's exponent, the conversion of u, the stencil)
    ("bf16x3", 3, 1 + 6 * 4 + 2 + 3),
    ("bf16x3", 0, 1 + 6),
])
def test_launch_count_per_solve(sem3d, tier, sweeps, expected):
    with sem3d.Plan(*N3, K, L3, C) as p:
        p.set_precision(tier, sweeps)
        f = torch.from_numpy(random_rhs(*N3, seed=600)).cuda()
        u = torch.empty_like(f)
        p.solve(f, u)  # workspace and first-use setup outside the count
        p.sync_check()
        n0 = p.launch_count()
        for _ in range(3):
            p.solve(f, u)
        p.sync_check()
        assert p.launch_count() - n0 == 3 * expected


def test_profile_counts_and_times(sem3d):
    with sem3d.Plan(*N3, K, L3, C) as p:
        p.set_precision("bf16x3", 3)
        f = torch.from_numpy(random_rhs(*N3, seed=601)).cuda()
        u = torch.empty_like(f)
        p.solve(f, u)
        p.sync_check()
        p.profile(True)
        n0 = p.launch_count()
        p.solve(f, u)
        p.solve(f, u)
        launches = p.launch_count() - n0
        got = {kind: p.profile_read(kind) for kind in ("tc_mode_product", "f64_mode_product", "stencil", "split",
                                                      "tc_x", "tc_y", "tc_z", "tc_f64_out", "f32_mode_product")}
        p.profile(False)
        p.sync_check()
    assert got["tc_mode_product"][0] == 2 * 24
    assert got["split"][0] == 2
    assert got["stencil"][0] == 2 * 5          # 2 double-FP32 + the fixed-point residual's 3 launches
    assert got["f64_mode_product"][0] == 0 and got["f32_mode_product"][0] == 0
    # per-pass classes partition the tensor-core launches
    assert (got["tc_x"][0] + got["tc_y"][0] + got["tc_z"][0] + got["tc_f64_out"][0]) == 2 * 24
    assert got["tc_f64_out"][0] == 2 * 4        # the last pass of each of the 4 solves
    assert launches == got["tc_mode_product"][0] + got["split"][0] + got["stencil"][0]
    for kind in ("tc_mode_product", "stencil", "split"):
        assert got[kind][1] > 0.0
