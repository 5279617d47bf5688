"""CPU-only checks of the C ABI: the library builds and loads, exports every
entry point include/sem3d.h declares, validates arguments, and its host FP64
setup (Newton GLL + Householder/QR eigensolver) agrees with the oracle
(Golub-Welsch GLL + LAPACK eigh) -- two independent routes to the same 1D
data.  No GPU compute is called here."""

import os
import re
import time

import numpy as np
import pytest

from oracle import sem_1d
from paper_2310_00226_gb300 import build, sem3d

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return sem3d.lib()


def _declared_symbols():
    with open(os.path.join(ROOT, "include", "sem3d.h")) as fh:
        text = fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sem3d_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol(L):
    declared = _declared_symbols()
    assert len(declared) >= 10
    for name in declared:
        assert hasattr(L, name), name
    assert sorted(declared) == sorted(sem3d.EXPORTS)


def test_setup_argument_validation(L):
    import ctypes
    h = ctypes.c_void_p()
    bad = [
        (8, 7, 7, 2, 1.0, 1.0, 1.0, 0.0),    # (n+1) % k != 0
        (7, 7, 7, 0, 1.0, 1.0, 1.0, 0.0),    # k = 0
        (7, 7, 7, 25, 1.0, 1.0, 1.0, 0.0),   # k too large
        (0, 7, 7, 1, 1.0, 1.0, 1.0, 0.0),    # n = 0
        (7, 7, 7, 2, -1.0, 1.0, 1.0, 0.0),   # L <= 0
        (7, 7, 7, 2, 1.0, 1.0, 1.0, -1e9),   # indefinite shift
        (7, 7, 7, 2, 1.0, 1.0, 1.0, float("nan")),
    ]
    for args in bad:
        st = L.sem3d_setup(*args, ctypes.byref(h))
        assert st == 1, (args, st)
        assert L.sem3d_last_error()
    assert L.sem3d_setup(7, 7, 7, 2, 1.0, 1.0, 1.0, 0.0, None) == 1
    assert L.sem3d_set_precision(None, 0, 1) == 1
    h = ctypes.c_void_p()
    # Neumann: (n-1) % k == 0, n > k and c > 0; an unknown boundary condition is rejected
    assert L.sem3d_setup_bc(8, 9, 9, 2, 1.0, 1.0, 1.0, 1.0, 1, ctypes.byref(h)) == 1
    assert L.sem3d_setup_bc(1, 9, 9, 2, 1.0, 1.0, 1.0, 1.0, 1, ctypes.byref(h)) == 1
    assert L.sem3d_setup_bc(9, 9, 9, 2, 1.0, 1.0, 1.0, 0.0, 1, ctypes.byref(h)) == 1
    assert b"c must be > 0" in L.sem3d_last_error()
    assert L.sem3d_setup_bc(7, 7, 7, 2, 1.0, 1.0, 1.0, 1.0, 2, ctypes.byref(h)) == 1
    assert L.sem3d_tuned_config(None, 0, None) == 1
    assert L.sem3d_inject_stall(None, 1) == 1
    assert L.sem3d_set_tuned_config(None, 0, 0) == 1
    assert L.sem3d_destroy(None) == 0


@pytest.mark.parametrize("n,k,Lb", [(1, 1, 1.0), (1, 2, 1.0), (7, 2, 1.0), (11, 3, 0.7), (39, 5, 2.0),
                                    (63, 2, 1.0), (191, 6, 2.0), (79, 20, 1.0)])
def test_host_axis_setup_matches_oracle(L, n, k, Lb):
    x, M, lam, T = sem3d.axis_info(n, k, Lb)
    s = sem_1d(k, (n + 1) // k, 0.0, Lb)
    np.testing.assert_allclose(x, s.x, rtol=0, atol=1e-14 * Lb)
    np.testing.assert_allclose(M, s.M, rtol=1e-13)
    np.testing.assert_allclose(lam, s.lam, rtol=5e-13 * max(1, n / 50), atol=1e-12)
    # Eigenvectors: same columns up to sign (both use the largest-entry-positive
    # convention, but compare through |<t_lib, M t_orc>| = 1 to be robust).
    G = np.abs(T.T @ (s.M[:, None] * s.T))
    np.testing.assert_allclose(np.diag(G), 1.0, atol=1e-11 * max(1, n / 50))


def test_host_axis_setup_headline_size(L):
    t0 = time.time()
    x, M, lam, T = sem3d.axis_info(999, 4, 1.0)
    dt = time.time() - t0
    assert abs(lam[0] - np.pi**2) < 1e-9
    # orthogonality in the M inner product: T^T M T = I
    G = T.T @ (M[:, None] * T)
    assert np.abs(G - np.eye(999)).max() < 1e-11
    assert dt < 120.0


def test_host_axis_setup_rejects_bad_args(L):
    with pytest.raises(sem3d.Sem3dError):
        sem3d.axis_info(8, 2, 1.0)
    with pytest.raises(sem3d.Sem3dError):
        sem3d.axis_info(7, 2, 0.0)
