"""Caller-owned device workspace (sem3d_workspace_size / sem3d_set_workspace).

A solve in a workspace the caller allocated (here a torch buffer) gives the
same result bit for bit as one in the plan's own workspace, in every tier.
set_workspace rejects a buffer smaller than sem3d_workspace_size or not
256-byte aligned; when a tier that needs more is selected later, the next
solve fails instead of writing past the caller's buffer.
"""

import numpy as np
import pytest

from paper_2310_00226_gb300.inputs import random_rhs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TIERS = [("fp64", 1), ("fp32", 2), ("tf32", 5), ("bf16x3", 3), ("f16x3", 3)]
N3, K, L3, C = (63, 39, 47), 2, (1.0, 1.0, 1.0), 3.0


@pytest.fixture(scope="module")
def sem3d():
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_2310_00226_gb300 import sem3d as mod
    mod.lib()
    return mod


@pytest.mark.parametrize("tier,sweeps", TIERS)
def test_caller_workspace_matches_plan_workspace(sem3d, tier, sweeps):
    f = torch.from_numpy(random_rhs(*N3, seed=500)).cuda()
    u_own, u_ws = torch.empty_like(f), torch.empty_like(f)
    with sem3d.Plan(*N3, K, L3, C) as p:
        p.set_precision(tier, sweeps)
        p.solve(f, u_own)
        p.sync_check()
    with sem3d.Plan(*N3, K, L3, C) as q:
        q.set_precision(tier, sweeps)
        nb = q.workspace_size()
        assert nb > 0 and nb % 256 == 0
        ws = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
        assert ws.data_ptr() % 256 == 0
        with pytest.raises(sem3d.Sem3dError):
            q.set_workspace(ws[: nb - 256])          # too small
        with pytest.raises(sem3d.Sem3dError):
            q.set_workspace(ws[16: nb + 16])         # misaligned
        q.set_workspace(ws[:nb])
        q.solve(f, u_ws)
        q.sync_check()
    assert torch.equal(u_own, u_ws)


def test_caller_workspace_too_small_for_a_later_tier(sem3d):
    f = torch.from_numpy(random_rhs(*N3, seed=501)).cuda()
    u = torch.empty_like(f)
    with sem3d.Plan(*N3, K, L3, C) as q:
        sizes = {}
        for tier, sweeps in TIERS:
            q.set_precision(tier, sweeps)
            sizes[tier] = q.workspace_size()
        small = min(sizes, key=sizes.get)
        large = max(sizes, key=sizes.get)
        assert sizes[large] > sizes[small]
        q.set_precision(small, dict(TIERS)[small])
        ws = torch.empty(sizes[small], dtype=torch.uint8, device="cuda")
        q.set_workspace(ws)
        q.solve(f, u)
        q.sync_check()
        q.set_precision(large, dict(TIERS)[large])
        with pytest.raises(sem3d.Sem3dError):
            q.solve(f, u)
        assert np.isfinite(u.cpu().numpy()).all()
