"""GPU parity of the Cahn-Hilliard BDF2 step (sem3d_ch_step / sem3d_ch_run)
against the oracle's dense solve of the same step (Section 3.5, Eqs. 19-20).

Tolerances (relative L-inf after the stated number of steps): FP64 tier 1e-11
(rounding of two spectral transforms per step), FP32 tier 1e-5, BF16x3 tier
2e-4 (no refinement inside a time step: the tier's own accuracy).
"""

import numpy as np
import pytest

from oracle import ch_step, sem_1d

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS, M, DT = 0.1, 1.0, 1e-5


@pytest.fixture(scope="module")
def sem3d():
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_2310_00226_gb300 import sem3d as mod
    mod.lib()
    return mod


def _setup(n3, k, seed):
    axes = [sem_1d(k, (n + 1) // k, 0.0, 1.0) for n in n3]
    rng = np.random.Generator(np.random.PCG64(seed))
    phi0 = rng.uniform(-0.6, 0.6, (n3[2], n3[1], n3[0]))
    return axes, phi0


def _oracle_run(phi_m, phi, axes, nsteps, S):
    sx, sy, sz = axes
    for _ in range(nsteps):
        phi_m, phi = phi, ch_step(phi, phi_m, sx, sy, sz, EPS, M, DT, S)
    return phi_m, phi


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32", 1e-5), ("bf16x3", 2e-4)])
@pytest.mark.parametrize("S", [0.0, 2.0])
def test_ch_step_matches_oracle(sem3d, prec, tol, S):
    n3, k = (7, 9, 11), 2
    axes, phi0 = _setup(n3, k, seed=4)
    _, ref1 = _oracle_run(phi0, phi0, axes, 1, S)
    ref5m, ref5 = _oracle_run(phi0, phi0, axes, 5, S)
    with sem3d.Plan(*n3, k, (1.0, 1.0, 1.0), 0.0) as p:
        p.set_precision(prec, 0)
        a = torch.from_numpy(phi0).cuda()
        out = torch.empty_like(a)
        p.ch_step(a, a, out, EPS, M, DT, S)
        p.sync_check()
        got1 = out.cpu().numpy()
        pm, pn = a.clone(), a.clone()
        p.ch_run(pm, pn, 5, EPS, M, DT, S)
        p.sync_check()
        got5, got5m = pn.cpu().numpy(), pm.cpu().numpy()
    rel = lambda x, y: float(np.abs(x - y).max() / np.abs(y).max())  # noqa: E731
    assert rel(got1, ref1) < tol
    assert rel(got5, ref5) < tol
    assert rel(got5m, ref5m) < tol


@pytest.mark.parametrize("nsteps", [1, 2, 3, 4, 5, 7])
def test_ch_run_equals_repeated_steps(sem3d, nsteps):
    # The graph-replayed run must reproduce step-by-step calls exactly (same
    # kernels, same order), for every residue of nsteps modulo the 3-buffer rotation.
    n3, k = (7, 7, 7), 2
    axes, phi0 = _setup(n3, k, seed=9)
    with sem3d.Plan(*n3, k, (1.0, 1.0, 1.0), 0.0) as p:
        p.set_precision("fp64", 0)
        a = torch.from_numpy(phi0).cuda()
        pm, pn = a.clone(), a.clone()
        for _ in range(nsteps):
            nxt = torch.empty_like(pn)
            p.ch_step(pn, pm, nxt, EPS, M, DT, 2.0)
            pm, pn = pn, nxt
        qm, qn = a.clone(), a.clone()
        p.ch_run(qm, qn, nsteps, EPS, M, DT, 2.0)
        p.sync_check()
        assert torch.equal(qn, pn)
        assert torch.equal(qm, pm)
