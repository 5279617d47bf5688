"""Python binding of the libsem3d C ABI (include/sem3d.h): argument marshalling only.

Every step of the solve runs in the library's CUDA kernels; this module only
converts torch tensors and streams into pointers.  It never falls back to
another implementation: if ``libsem3d.so`` is missing, loading raises.

Arrays are torch tensors of dtype float64 on a CUDA device, contiguous, of
shape (nz, ny, nx) (x fastest, the layout of the C ABI) or flat.
"""

from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libsem3d.so")

SEM3D_OK = 0
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "CUDA", 3: "OOM", 4: "NOT_CONVERGED", 5: "TIMEOUT", 6: "UNSUPPORTED"}
PRECISIONS = {"fp64": 0, "fp32": 1, "tf32": 2, "bf16": 4, "bf16x3": 5, "f16x3": 6}

#: Every entry point declared in include/sem3d.h.
EXPORTS = (
    "sem3d_setup",
    "sem3d_setup_bc",
    "sem3d_set_precision",
    "sem3d_set_residual",
    "sem3d_set_exact_residual",
    "sem3d_exact_residual_kind",
    "sem3d_workspace_size",
    "sem3d_set_workspace",
    "sem3d_solve",
    "sem3d_solve_host",
    "sem3d_solve_host_wait",
    "sem3d_solve_batched",
    "sem3d_apply",
    "sem3d_pcg",
    "sem3d_ch_step",
    "sem3d_ch_run",
    "sem3d_get_nodes",
    "sem3d_get_eigs",
    "sem3d_axis_info",
    "sem3d_sync_check",
    "sem3d_profile",
    "sem3d_profile_read",
    "sem3d_launch_count",
    "sem3d_tuned_config",
    "sem3d_set_tuned_config",
    "sem3d_tc_config",
    "sem3d_set_tc_config",
    "sem3d_inject_stall",
    "sem3d_solve_fp64_static",
    "sem3d_destroy",
    "sem3d_last_error",
)

_lib = None


class Sem3dError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def lib() -> ctypes.CDLL:
    """Load libsem3d.so (built by paper_2310_00226_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError(f"libsem3d.so not found at {_LIB_PATH}; run paper_2310_00226_gb300.build.build()")
    L = ctypes.CDLL(_LIB_PATH)
    c_int, c_double, c_void_p, c_size_t = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t
    L.sem3d_setup.argtypes = [c_int, c_int, c_int, c_int, c_double, c_double, c_double, c_double,
                              ctypes.POINTER(c_void_p)]
    L.sem3d_setup_bc.argtypes = [c_int, c_int, c_int, c_int, c_double, c_double, c_double, c_double, c_int,
                                 ctypes.POINTER(c_void_p)]
    L.sem3d_set_precision.argtypes = [c_void_p, c_int, c_int]
    L.sem3d_set_residual.argtypes = [c_void_p, c_int]
    L.sem3d_set_exact_residual.argtypes = [c_void_p, c_int]
    L.sem3d_exact_residual_kind.argtypes = [c_void_p, ctypes.POINTER(c_int)]
    L.sem3d_workspace_size.argtypes = [c_void_p, ctypes.POINTER(c_size_t)]
    L.sem3d_set_workspace.argtypes = [c_void_p, c_void_p, c_size_t]
    L.sem3d_solve.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p]
    L.sem3d_solve_host.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p]
    L.sem3d_solve_host_wait.argtypes = [c_void_p, c_void_p]
    L.sem3d_apply.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p]
    L.sem3d_solve_batched.argtypes = [c_int, ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p),
                                      ctypes.POINTER(c_void_p), c_void_p]
    L.sem3d_pcg.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_double, c_int, ctypes.POINTER(c_int),
                            ctypes.POINTER(c_double), c_void_p]
    L.sem3d_ch_step.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_double, c_double, c_double, c_double,
                                c_void_p]
    L.sem3d_ch_run.argtypes = [c_void_p, c_void_p, c_void_p, c_int, c_double, c_double, c_double, c_double, c_void_p]
    L.sem3d_get_nodes.argtypes = [c_void_p, c_int, c_void_p]
    L.sem3d_get_eigs.argtypes = [c_void_p, c_int, c_void_p, c_void_p]
    L.sem3d_axis_info.argtypes = [c_int, c_int, c_double, c_void_p, c_void_p, c_void_p, c_void_p]
    L.sem3d_sync_check.argtypes = [c_void_p, c_void_p]
    L.sem3d_profile.argtypes = [c_void_p, c_int]
    L.sem3d_profile_read.argtypes = [c_void_p, c_int, ctypes.POINTER(ctypes.c_longlong),
                                     ctypes.POINTER(ctypes.c_double)]
    L.sem3d_launch_count.argtypes = [c_void_p, ctypes.POINTER(ctypes.c_ulonglong)]
    L.sem3d_tuned_config.argtypes = [c_void_p, c_int, ctypes.POINTER(c_int)]
    L.sem3d_set_tuned_config.argtypes = [c_void_p, c_int, c_int]
    L.sem3d_tc_config.argtypes = [c_void_p, c_int, ctypes.POINTER(c_int)]
    L.sem3d_set_tc_config.argtypes = [c_void_p, c_int, c_int]
    L.sem3d_inject_stall.argtypes = [c_void_p, c_int]
    L.sem3d_solve_fp64_static.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p]
    L.sem3d_destroy.argtypes = [c_void_p]
    L.sem3d_last_error.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name != "sem3d_last_error":
            getattr(L, name).restype = c_int
    _lib = L
    return L


def _check(status: int, where: str):
    if status != SEM3D_OK:
        raise Sem3dError(status, where, lib().sem3d_last_error().decode())


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _dev_ptr(t, n: int, name: str) -> int:
    import torch
    if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous float64 CUDA tensor")
    if t.numel() != n:
        raise ValueError(f"{name} has {t.numel()} elements, expected {n}")
    return t.data_ptr()


def _host_ptr(t, n: int, name: str) -> int:
    import torch
    if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous float64 CPU tensor (pinned for asynchronous copies)")
    if t.numel() != n:
        raise ValueError(f"{name} has {t.numel()} elements, expected {n}")
    return t.data_ptr()


def axis_info(n: int, k: int, L: float = 1.0):
    """Host-only 1D axis data as sem3d_setup builds it: (x, M, lambda, T)."""
    x, M, lam = np.empty(n), np.empty(n), np.empty(n)
    T = np.empty((n, n), order="F")
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    _check(lib().sem3d_axis_info(n, k, float(L), ptr(x), ptr(M), ptr(lam), ptr(T)), "sem3d_axis_info")
    return x, M, lam, T


def solve_batched(plans, fs, us, stream=None):
    """sem3d_solve_batched over lists of plans and float64 CUDA tensors."""
    n = len(plans)
    if not (n == len(fs) == len(us)):
        raise ValueError("plans, fs and us must have the same length")
    H = (ctypes.c_void_p * n)(*[p._h.value for p in plans])
    F = (ctypes.c_void_p * n)(*[_dev_ptr(f, p.numel, "f") for p, f in zip(plans, fs)])
    U = (ctypes.c_void_p * n)(*[_dev_ptr(u, p.numel, "u") for p, u in zip(plans, us)])
    _check(lib().sem3d_solve_batched(n, H, F, U, ctypes.c_void_p(_stream_ptr(stream))), "sem3d_solve_batched")


class Plan:
    """A libsem3d plan (sem3d_setup ... sem3d_destroy)."""

    BCS = {"dirichlet": 0, "neumann": 1}

    def __init__(self, nx: int, ny: int, nz: int, k: int, L=(1.0, 1.0, 1.0), c: float = 0.0, bc: str = "dirichlet"):
        h = ctypes.c_void_p()
        _check(lib().sem3d_setup_bc(nx, ny, nz, k, float(L[0]), float(L[1]), float(L[2]), float(c), self.BCS[bc],
                                    ctypes.byref(h)), "sem3d_setup_bc")
        self._h = h
        self.bc = bc
        self.shape = (nz, ny, nx)
        self.n = (nx, ny, nz)
        self.k = k
        self.c = c

    @property
    def numel(self) -> int:
        nx, ny, nz = self.n
        return nx * ny * nz

    def set_precision(self, precision: str = "fp64", sweeps: int = 1):
        _check(lib().sem3d_set_precision(self._h, PRECISIONS[precision], int(sweeps)), "sem3d_set_precision")

    RESIDUALS = {"fp64": 0, "mixed": 1, "df": 2}

    def set_residual(self, mode: str = "mixed"):
        _check(lib().sem3d_set_residual(self._h, self.RESIDUALS[mode]), "sem3d_set_residual")

    EXACT = {"fixed": 0, "fp64": 1}

    def set_exact_residual(self, kind: str = "fixed"):
        """Arithmetic of the split tiers' FP64-accurate residuals: "fixed"
        (64-bit integer fixed point) or "fp64" (FP64 FMAs)."""
        _check(lib().sem3d_set_exact_residual(self._h, self.EXACT[kind]), "sem3d_set_exact_residual")

    def exact_residual_kind(self) -> str:
        k = ctypes.c_int()
        _check(lib().sem3d_exact_residual_kind(self._h, ctypes.byref(k)), "sem3d_exact_residual_kind")
        return {v: n for n, v in self.EXACT.items()}[k.value]

    def workspace_size(self) -> int:
        b = ctypes.c_size_t()
        _check(lib().sem3d_workspace_size(self._h, ctypes.byref(b)), "sem3d_workspace_size")
        return b.value

    def set_workspace(self, buf):
        _check(lib().sem3d_set_workspace(self._h, ctypes.c_void_p(buf.data_ptr()), buf.numel() * buf.element_size()),
               "sem3d_set_workspace")

    def solve(self, f, u, stream=None):
        _check(lib().sem3d_solve(self._h, ctypes.c_void_p(_dev_ptr(f, self.numel, "f")),
                                 ctypes.c_void_p(_dev_ptr(u, self.numel, "u")), ctypes.c_void_p(_stream_ptr(stream))),
               "sem3d_solve")

    def solve_host(self, f_host, u_host, stream=None):
        """Solve with host (pinned) tensors; pipelined with the plan's other solve_host calls.
        Results are complete after solve_host_wait(stream) and a synchronisation of the stream."""
        _check(lib().sem3d_solve_host(self._h, ctypes.c_void_p(_host_ptr(f_host, self.numel, "f_host")),
                                      ctypes.c_void_p(_host_ptr(u_host, self.numel, "u_host")),
                                      ctypes.c_void_p(_stream_ptr(stream))), "sem3d_solve_host")

    def solve_host_wait(self, stream=None):
        _check(lib().sem3d_solve_host_wait(self._h, ctypes.c_void_p(_stream_ptr(stream))), "sem3d_solve_host_wait")

    def apply(self, u, Au, stream=None):
        _check(lib().sem3d_apply(self._h, ctypes.c_void_p(_dev_ptr(u, self.numel, "u")),
                                 ctypes.c_void_p(_dev_ptr(Au, self.numel, "Au")), ctypes.c_void_p(_stream_ptr(stream))),
               "sem3d_apply")

    def pcg(self, V, f, u, rtol: float = 1e-10, maxit: int = 200, stream=None, check: bool = True):
        """PCG for -Lap u + V u = f preconditioned by this plan's solve; returns (iters, relres)."""
        it, rr = ctypes.c_int(), ctypes.c_double()
        st = lib().sem3d_pcg(self._h, ctypes.c_void_p(_dev_ptr(V, self.numel, "V")),
                             ctypes.c_void_p(_dev_ptr(f, self.numel, "f")), ctypes.c_void_p(_dev_ptr(u, self.numel, "u")),
                             float(rtol), int(maxit), ctypes.byref(it), ctypes.byref(rr),
                             ctypes.c_void_p(_stream_ptr(stream)))
        if check:
            _check(st, "sem3d_pcg")
        return it.value, rr.value

    def ch_step(self, phi_n, phi_nm1, phi_np1, eps: float, m: float, dt: float, S: float = 0.0, stream=None):
        _check(lib().sem3d_ch_step(self._h, ctypes.c_void_p(_dev_ptr(phi_n, self.numel, "phi_n")),
                                   ctypes.c_void_p(_dev_ptr(phi_nm1, self.numel, "phi_nm1")),
                                   ctypes.c_void_p(_dev_ptr(phi_np1, self.numel, "phi_np1")), float(eps), float(m),
                                   float(dt), float(S), ctypes.c_void_p(_stream_ptr(stream))), "sem3d_ch_step")

    def ch_run(self, phi_nm1, phi_n, nsteps: int, eps: float, m: float, dt: float, S: float = 0.0, stream=None):
        _check(lib().sem3d_ch_run(self._h, ctypes.c_void_p(_dev_ptr(phi_nm1, self.numel, "phi_nm1")),
                                  ctypes.c_void_p(_dev_ptr(phi_n, self.numel, "phi_n")), int(nsteps), float(eps),
                                  float(m), float(dt), float(S), ctypes.c_void_p(_stream_ptr(stream))), "sem3d_ch_run")

    def sync_check(self, stream=None):
        _check(lib().sem3d_sync_check(self._h, ctypes.c_void_p(_stream_ptr(stream))), "sem3d_sync_check")

    KERNEL_CLASSES = {"tc_mode_product": 0, "f64_mode_product": 1, "stencil": 2, "split": 3,
                      "tc_x": 4, "tc_y": 5, "tc_z": 6, "tc_f64_out": 7, "f32_mode_product": 8}

    def profile(self, enable: bool = True):
        _check(lib().sem3d_profile(self._h, 1 if enable else 0), "sem3d_profile")

    def profile_read(self, kind: str):
        """(launches, total_ms) of one kernel class since profiling was enabled."""
        n, ms = ctypes.c_longlong(), ctypes.c_double()
        _check(lib().sem3d_profile_read(self._h, self.KERNEL_CLASSES[kind], ctypes.byref(n), ctypes.byref(ms)),
               "sem3d_profile_read")
        return n.value, ms.value

    def launch_count(self) -> int:
        n = ctypes.c_ulonglong()
        _check(lib().sem3d_launch_count(self._h, ctypes.byref(n)), "sem3d_launch_count")
        return n.value

    def tuned_config(self, axis: int) -> int:
        """FP32 kernel configuration the autotuner picked for the pass along axis."""
        c = ctypes.c_int()
        _check(lib().sem3d_tuned_config(self._h, axis, ctypes.byref(c)), "sem3d_tuned_config")
        return c.value

    def set_tuned_config(self, axis: int, config: int):
        """Pin an FP32 kernel configuration for this plan's pass shape along axis."""
        _check(lib().sem3d_set_tuned_config(self._h, axis, config), "sem3d_set_tuned_config")

    def tc_config(self, axis: int) -> int:
        """Tensor-core kernel (0 = single CTA, 1 = CTA pair) chosen for the pass along axis."""
        c = ctypes.c_int()
        _check(lib().sem3d_tc_config(self._h, axis, ctypes.byref(c)), "sem3d_tc_config")
        return c.value

    def set_tc_config(self, axis: int, config: int):
        """Pin the tensor-core kernel (0 = single CTA, 1 = CTA pair) for this plan's pass shape along axis."""
        _check(lib().sem3d_set_tc_config(self._h, axis, config), "sem3d_set_tc_config")

    def nodes(self, axis: int) -> np.ndarray:
        x = np.empty(self.n[axis])
        _check(lib().sem3d_get_nodes(self._h, axis, x.ctypes.data_as(ctypes.c_void_p)), "sem3d_get_nodes")
        return x

    def eigs(self, axis: int, with_vectors: bool = False):
        n = self.n[axis]
        lam = np.empty(n)
        T = np.empty((n, n), order="F") if with_vectors else None
        _check(lib().sem3d_get_eigs(self._h, axis, lam.ctypes.data_as(ctypes.c_void_p),
                                    T.ctypes.data_as(ctypes.c_void_p) if T is not None else None), "sem3d_get_eigs")
        return (lam, T) if with_vectors else lam

    def close(self):
        if getattr(self, "_h", None):
            _check(lib().sem3d_destroy(self._h), "sem3d_destroy")
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
