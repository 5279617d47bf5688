"""The allocation-free FP64 solve (sem3d_solve_fp64_static) against sem3d_solve.

Callers that cannot let the library call cudaMalloc (their device memory
belongs to another allocator, or they must avoid the device synchronisation an
allocation may cause) use sem3d_solve_fp64_static, whose scratch is a fixed
device array inside the library.  This test calls it twice in a row through
the C ABI and checks each result against the regular entry point, with the
tolerance of the FP64 parity tests (relative L-infinity 1e-12).  It lives in a
file that pytest collects last and passes both alone and after other tests.
"""

import ctypes

import numpy as np
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


@pytest.mark.parametrize("n3,k,c", [((63, 39, 47), 2, 3.0), ((79, 79, 79), 4, 1.0)])
def test_static_scratch_solve_matches_sem3d_solve(sem3d, n3, k, c):
    L = sem3d.lib()
    with sem3d.Plan(*n3, k, (1.0, 0.8, 1.2), c) as p:
        p.set_precision("fp64", 1)
        f = torch.from_numpy(random_rhs(*n3, seed=11)).cuda()
        u_ref = torch.empty_like(f)
        p.solve(f, u_ref)
        p.sync_check()
        stream = torch.cuda.current_stream().cuda_stream
        for _ in range(2):
            u = torch.full_like(f, float("nan"))
            st = L.sem3d_solve_fp64_static(p._h, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(u.data_ptr()),
                                           ctypes.c_void_p(stream))
            assert st == 0, L.sem3d_last_error()
            p.sync_check()
            assert torch.isfinite(u).all()
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
