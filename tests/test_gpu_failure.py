"""Failure detection on the GPU without a GPU fault.

Every wait inside the tensor-core kernel is bounded (1 s on the global timer)
and records SEM3D_ERR_TIMEOUT in the plan's device error word when it expires.
sem3d_inject_stall makes the next tensor-core launch issue no operand loads, so
the MMA warp waits on a barrier that nothing arms: the wait must expire, the
kernel must return (releasing its tensor memory), sem3d_sync_check must report
the timeout, and the same plan must then solve correctly.
"""

import numpy as np
import pytest

from oracle import refined_solve, sem_1d
from paper_2310_00226_gb300.inputs import batched_helmholtz, random_rhs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TIMEOUT = 5  # SEM3D_ERR_TIMEOUT


@pytest.fixture(scope="module")
def sem3d():
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_2310_00226_gb300 import sem3d as mod
    mod.lib()
    return mod


@pytest.mark.parametrize("tier,sweeps", [("bf16x3", 3), ("f16x3", 3), ("tf32", 5)])
def test_expired_wait_is_reported_and_the_plan_recovers(sem3d, tier, sweeps):
    n3, k = (63, 31, 47), 2
    axes = [sem_1d(k, (n + 1) // k, 0.0, 1.0) for n in n3]
    F = random_rhs(*n3, seed=17)
    ref = refined_solve(F, *axes, 1.0, sweeps=1)
    with sem3d.Plan(*n3, k, (1.0, 1.0, 1.0), 1.0) as p:
        f = torch.from_numpy(F).cuda()
        u = torch.empty_like(f)
        p.set_precision(tier, 0)
        p.solve(f, u)              # warm-up: workspace and kernels loaded
        p.sync_check()
        assert sem3d.lib().sem3d_inject_stall(p._h, 1) == 0
        p.solve(f, u)              # the first pass's producer stalls
        with pytest.raises(sem3d.Sem3dError) as exc:
            p.sync_check()
        assert exc.value.status == TIMEOUT
        # the error word was cleared and the context is usable: a normal refined solve
        p.set_precision(tier, sweeps)
        p.solve(f, u)
        p.sync_check()
        err = float(np.abs(u.cpu().numpy() - ref).max() / np.abs(ref).max())
        assert err < 1e-12, err


def test_injection_is_consumed_once(sem3d):
    with sem3d.Plan(15, 15, 15, 2, (1.0, 1.0, 1.0), 1.0) as p:
        p.set_precision("bf16x3", 1)
        f = torch.ones(15 ** 3, dtype=torch.float64, device="cuda")
        u = torch.empty_like(f)
        assert sem3d.lib().sem3d_inject_stall(p._h, 1) == 0
        assert sem3d.lib().sem3d_inject_stall(p._h, 0) == 0   # cancelled before any launch
        p.solve(f, u)
        p.sync_check()                                        # no timeout


@pytest.mark.parametrize("variant", [0, 1])
def test_expired_wait_in_each_split_tier_kernel(sem3d, variant):
    # the one-CTA kernel (0) and the CTA-pair kernel (1) pinned in turn
    n3, k = (63, 31, 47), 2
    axes = [sem_1d(k, (n + 1) // k, 0.0, 1.0) for n in n3]
    F = random_rhs(*n3, seed=18)
    ref = refined_solve(F, *axes, 1.0, sweeps=1)
    with sem3d.Plan(*n3, k, (1.0, 1.0, 1.0), 1.0) as p:
        for ax in range(3):
            p.set_tc_config(ax, variant)
        p.set_precision("bf16x3", 0)
        f = torch.from_numpy(F).cuda()
        u = torch.empty_like(f)
        p.solve(f, u)
        p.sync_check()
        assert sem3d.lib().sem3d_inject_stall(p._h, 1) == 0
        p.solve(f, u)
        with pytest.raises(sem3d.Sem3dError) as exc:
            p.sync_check()
        assert exc.value.status == TIMEOUT
        p.set_precision("bf16x3", 3)
        p.solve(f, u)
        p.sync_check()
        assert float(np.abs(u.cpu().numpy() - ref).max() / np.abs(ref).max()) < 1e-12


def test_expired_wait_in_a_grouped_batch(sem3d):
    # one persistent CTA-pair launch per pass over all problems: its producer
    # stalls, the waits expire, the batch reports the timeout through the first
    # plan, and the next batch solves correctly
    probs = batched_helmholtz(count=4, seed=9, sizes=(31, 47, 63), degrees=(2, 4))
    plans, fs, us, refs = [], [], [], []
    try:
        for pr in probs:
            p = sem3d.Plan(*pr["n3"], pr["k"], (1.0, 1.0, 1.0), pr["c"])
            p.set_precision("bf16x3", 0)
            F = random_rhs(*pr["n3"], seed=pr["seed"])
            axes = [sem_1d(pr["k"], (n + 1) // pr["k"], 0.0, 1.0) for n in pr["n3"]]
            refs.append(refined_solve(F, *axes, pr["c"], sweeps=1))
            plans.append(p)
            fs.append(torch.from_numpy(F).cuda())
            us.append(torch.empty_like(fs[-1]))
        sem3d.solve_batched(plans, fs, us)
        plans[0].sync_check()
        assert sem3d.lib().sem3d_inject_stall(plans[0]._h, 1) == 0
        sem3d.solve_batched(plans, fs, us)
        with pytest.raises(sem3d.Sem3dError) as exc:
            plans[0].sync_check()
        assert exc.value.status == TIMEOUT
        for p in plans:
            p.set_precision("bf16x3", 3)
        sem3d.solve_batched(plans, fs, us)
        plans[0].sync_check()
        for u, ref in zip(us, refs):
            assert float(np.abs(u.cpu().numpy() - ref).max() / np.abs(ref).max()) < 1e-12
    finally:
        for p in plans:
            p.close()
