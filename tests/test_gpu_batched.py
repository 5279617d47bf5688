"""GPU parity of sem3d_solve_batched against the oracle, problem by problem.

Grouped paths: every plan SEM3D_FP32 with the same sweeps (one FP32 launch
per pass for all problems), or every plan in one split tier (BF16x3 / BF16)
with the same sweeps and residual schedule (one persistent CTA-pair tcgen05
launch per pass for all problems, per-problem tensor maps in a device table).
Stream path: mixed tiers.  Tolerance: relative L-inf 1e-12 after refinement
(2 sweeps FP32, 3 sweeps BF16x3, 1 sweep FP64).  The grouped tensor-core
path issues the same MMAs as a plan's own solve, so its results must be
bit-identical to sem3d_solve of each plan.
"""

import numpy as np
import pytest

from oracle import refined_solve, sem_1d
from paper_2310_00226_gb300.inputs import batched_helmholtz, random_rhs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sem3d():
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_2310_00226_gb300 import sem3d as mod
    mod.lib()
    return mod


def _problems():
    # the batched workload's generator with small sizes (the oracle solves each in < 1 s)
    return batched_helmholtz(count=7, seed=77, sizes=(7, 11, 15, 23, 31, 47), degrees=(2, 3, 4, 6))


def _refs(probs):
    refs = []
    for pr in probs:
        n3, k, c = pr["n3"], pr["k"], pr["c"]
        axes = [sem_1d(k, (n + 1) // k, 0.0, 1.0) for n in n3]
        F = random_rhs(*n3, seed=pr["seed"])
        refs.append((F, refined_solve(F, *axes, c, sweeps=1)))
    return refs


@pytest.mark.parametrize("mode", ["grouped_fp32", "grouped_fp32_mixed_tiles", "streams_mixed",
                                  "grouped_bf16x3_mixed", "grouped_bf16x3_fp64", "grouped_bf16x3_df"])
def test_batched_matches_oracle(sem3d, mode):
    probs = _problems()
    refs = _refs(probs)
    plans, fs, us = [], [], []
    try:
        for q, pr in enumerate(probs):
            p = sem3d.Plan(*pr["n3"], pr["k"], (1.0, 1.0, 1.0), pr["c"])
            if mode.startswith("grouped_fp32"):
                p.set_precision("fp32", 2)
                if mode == "grouped_fp32_mixed_tiles":
                    # one grouped launch runs problems with different tile shapes
                    for a in range(3):
                        p.set_tuned_config(a, (q + a) % 6)
            elif mode.startswith("grouped_bf16x3"):
                p.set_precision("bf16x3", 3)
                p.set_residual(mode.split("_")[-1])
            else:
                p.set_precision(*[("fp32", 2), ("bf16x3", 3), ("fp64", 1), ("tf32", 5)][q % 4])
            plans.append(p)
            fs.append(torch.from_numpy(refs[q][0]).cuda())
            us.append(torch.full_like(fs[-1], float("nan")))
        for _ in range(2):  # twice: the staging area is reused
            sem3d.solve_batched(plans, fs, us)
            plans[0].sync_check()
            for q in range(len(probs)):
                got = us[q].cpu().numpy()
                ref = refs[q][1]
                assert np.abs(got - ref).max() / np.abs(ref).max() < 1e-12, (mode, q, probs[q])
    finally:
        for p in plans:
            p.close()


def test_batched_rejects_duplicate_plans(sem3d):
    with sem3d.Plan(7, 7, 7, 2) as p:
        f = torch.zeros(343, dtype=torch.float64, device="cuda")
        u = torch.empty_like(f)
        with pytest.raises(sem3d.Sem3dError):
            sem3d.solve_batched([p, p], [f, f], [u, u])


@pytest.mark.parametrize("tier,sweeps,residual", [("bf16x3", 3, "mixed"), ("bf16x3", 2, "fp64"), ("bf16x3", 2, "df"),
                                                  ("bf16", 0, "mixed"), ("bf16", 2, "mixed")])
def test_grouped_tensor_core_batch_is_bit_identical_to_single_solves(sem3d, tier, sweeps, residual):
    # Problems large enough for several pair tiles, N tiles and K blocks each,
    # of uneven n and k; the grouped launches must reproduce each plan's solve.
    probs = batched_helmholtz(count=6, seed=5, sizes=(63, 127, 191, 255), degrees=(2, 4))
    plans, fs, us, ref = [], [], [], []
    try:
        for pr in probs:
            p = sem3d.Plan(*pr["n3"], pr["k"], (1.0, 1.0, 1.0), pr["c"])
            p.set_precision(tier, sweeps)
            p.set_residual(residual)
            f = torch.from_numpy(random_rhs(*pr["n3"], seed=pr["seed"])).cuda()
            u = torch.empty_like(f)
            p.solve(f, u)
            p.sync_check()
            plans.append(p)
            fs.append(f)
            ref.append(u.cpu().numpy())
            us.append(torch.full_like(f, float("nan")))
        for _ in range(2):
            sem3d.solve_batched(plans, fs, us)
            plans[0].sync_check()
            for q in range(len(probs)):
                got = us[q].cpu().numpy()
                assert np.array_equal(got, ref[q]), (tier, q, probs[q], float(np.abs(got - ref[q]).max()))
    finally:
        for p in plans:
            p.close()


def test_grouped_neumann_batch_is_bit_identical_to_single_solves(sem3d):
    # Neumann plans (every GLL node kept, n = Ne*k + 1) take the grouped
    # tensor-core path with FP64 residuals in every sweep (per-row stencil);
    # sizes give ragged M, N and K tiles.
    shapes = [((129, 65, 97), 4, 2.0), ((97, 97, 33), 2, 1.0), ((41, 161, 81), 4, 5.0)]
    plans, fs, us, ref = [], [], [], []
    try:
        for q, (n3, k, c) in enumerate(shapes):
            p = sem3d.Plan(*n3, k, (1.0, 1.0, 1.0), c, bc="neumann")
            p.set_precision("bf16x3", 3)
            f = torch.from_numpy(random_rhs(*n3, seed=90 + q)).cuda()
            u = torch.empty_like(f)
            p.solve(f, u)
            p.sync_check()
            plans.append(p)
            fs.append(f)
            ref.append(u.cpu().numpy())
            us.append(torch.full_like(f, float("nan")))
        sem3d.solve_batched(plans, fs, us)
        plans[0].sync_check()
        for q in range(len(shapes)):
            assert np.array_equal(us[q].cpu().numpy(), ref[q]), q
    finally:
        for p in plans:
            p.close()
