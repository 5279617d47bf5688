"""The allocation-free FP64 solve (sem3d_solve_fp64_static) against sem3d_solve.

Callers that cannot let the library call cudaMalloc (their device memory
belongs to another allocator, or they must avoid the device synchronisation an
allocation may cause) use sem3d_solve_fp64_static, whose scratch is a fixed
device array inside the library.  These tests call it twice in a row through
the C ABI and check each result against the regular entry point, with the
tolerance of the FP64 parity tests (relative L-infinity 1e-12); they check
that a call on a plan that never had a workspace leaves the device's free
memory unchanged (no allocation), and that a plan set to another precision
still gets the FP64 result with the plan's sweep count.  The file is collected
last and its tests pass both alone and after the other tests.
"""

import ctypes

import pytest

from paper_2310_00226_gb300.inputs import random_rhs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def sem3d():
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_2310_00226_gb300 import sem3d as mod
    mod.lib()
    return mod


def _rel(a, b):
    return float((a - b).abs().max() / b.abs().max())


def _static_solve(L, plan, f, u):
    stream = torch.cuda.current_stream().cuda_stream
    st = L.sem3d_solve_fp64_static(plan._h, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(u.data_ptr()),
                                   ctypes.c_void_p(stream))
    assert st == 0, L.sem3d_last_error()


def _reference(sem3d, n3, k, box, c, sweeps, f):
    with sem3d.Plan(*n3, k, box, c) as q:
        q.set_precision("fp64", sweeps)
        u = torch.empty_like(f)
        q.solve(f, u)
        q.sync_check()
    return u


@pytest.mark.parametrize("n3,k,c", [((63, 39, 47), 2, 3.0), ((79, 79, 79), 4, 1.0)])
def test_static_scratch_solve_matches_sem3d_solve(sem3d, n3, k, c):
    L = sem3d.lib()
    box = (1.0, 0.8, 1.2)
    f = torch.from_numpy(random_rhs(*n3, seed=11)).cuda()
    u_ref = _reference(sem3d, n3, k, box, c, 1, f)
    with sem3d.Plan(*n3, k, box, c) as p:
        p.set_precision("fp64", 1)
        for _ in range(2):
            u = torch.full_like(f, float("nan"))
            _static_solve(L, p, f, u)
            p.sync_check()
            assert torch.isfinite(u).all()
            assert _rel(u, u_ref) <= TOL


def test_static_scratch_solve_allocates_nothing(sem3d):
    """A plan that never ran sem3d_solve has no workspace; two static solves on
    it must leave the device's free memory exactly where it was."""
    L = sem3d.lib()
    n3, k, c, box = (47, 55, 63), 4, 2.0, (1.0, 1.0, 1.0)
    f = torch.from_numpy(random_rhs(*n3, seed=5)).cuda()
    u_ref = _reference(sem3d, n3, k, box, c, 1, f)
    u1, u2 = torch.empty_like(f), torch.empty_like(f)
    # a first static call on another plan: the library's module and its scratch
    # array are resident before the measurement starts
    with sem3d.Plan(31, 31, 31, 4, box, 0.0) as w:
        fw = torch.ones(31**3, dtype=torch.float64, device="cuda")
        uw = torch.empty_like(fw)
        _static_solve(L, w, fw, uw)
        w.sync_check()
    with sem3d.Plan(*n3, k, box, c) as p:   # default mode FP64, 1 sweep; no workspace yet
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        _static_solve(L, p, f, u1)
        _static_solve(L, p, f, u2)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        p.sync_check()
        assert free1 == free0, f"free device memory changed by {free0 - free1} bytes"
        ws = ctypes.c_size_t(0)
        assert L.sem3d_workspace_size(p._h, ctypes.byref(ws)) == 0 and ws.value > 2 * 1024 * 1024
        assert _rel(u1, u_ref) <= TOL and _rel(u2, u_ref) <= TOL


def test_static_scratch_solve_ignores_the_plan_precision(sem3d):
    """A plan set to BF16x3 with 3 sweeps: the static solve runs the FP64 tier
    with those 3 sweeps, i.e. sem3d_solve after set_precision('fp64', 3)."""
    L = sem3d.lib()
    n3, k, c, box = (63, 47, 55), 4, 1.0, (1.0, 1.0, 1.0)
    f = torch.from_numpy(random_rhs(*n3, seed=9)).cuda()
    u_ref = _reference(sem3d, n3, k, box, c, 3, f)
    with sem3d.Plan(*n3, k, box, c) as p:
        p.set_precision("bf16x3", 3)
        for _ in range(2):
            u = torch.full_like(f, float("nan"))
            _static_solve(L, p, f, u)
            p.sync_check()
            assert _rel(u, u_ref) <= TOL


def test_static_scratch_solve_rejects_grids_above_limit(sem3d):
    L = sem3d.lib()
    # 81^3 = 531441 > 524288 unknowns
    with sem3d.Plan(81, 81, 81, 2, (1.0, 1.0, 1.0), 0.0) as p:
        f = torch.zeros(81**3, dtype=torch.float64, device="cuda")
        u = torch.empty_like(f)
        st = L.sem3d_solve_fp64_static(p._h, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(u.data_ptr()),
                                       ctypes.c_void_p(0))
        assert st == 1
        assert b"524288" in L.sem3d_last_error()
