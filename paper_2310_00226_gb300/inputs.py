"""Seeded synthetic inputs shared by the tests, the smoke check and the bench.

This module holds none of the solver's arithmetic: only the right-hand sides
(manufactured solutions and seeded noise) evaluated at node coordinates that
the caller passes in, and the sizes of the standard workloads.  Arrays are
(nz, ny, nx), C-contiguous, so the flat index is i + nx*(j + ny*l).

Manufactured solutions (all vanish on the boundary of their box, so they are
homogeneous-Dirichlet data):

* ``sine_123``: u = sin(pi x) sin(2 pi y) sin(3 pi z) on [0,1]^3,
  -Lap u = 14 pi^2 u  (the Q^2, n = 63 correctness workload, c = 0).
* ``exp_sine``: u = e^x sin(pi x) sin(pi y) sin(pi z) on [0,1]^3 with c = 1:
  -Lap u + u = e^x sin(pi y) sin(pi z) (3 pi^2 sin(pi x) - 2 pi cos(pi x))
  (the Q^4, n = 999 headline workload).
* ``table1_dirichlet``: u_D* of Section 3.1 on [-1,1]^3 with alpha = 1.
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

PI = math.pi


def _outer3(fx, fy, fz) -> np.ndarray:
    """(nz, ny, nx) array fz[l] * fy[j] * fx[i]."""
    return (np.asarray(fz)[:, None, None] * np.asarray(fy)[None, :, None]) * np.asarray(fx)[None, None, :]


def sine_123(x, y, z):
    """Returns (u, f) for -Lap u = f, u = sin(pi x) sin(2 pi y) sin(3 pi z)."""
    u = _outer3(np.sin(PI * x), np.sin(2 * PI * y), np.sin(3 * PI * z))
    return u, 14.0 * PI**2 * u


def exp_sine(x, y, z, c: float = 1.0):
    """Returns (u, f) for -Lap u + c u = f, u = e^x sin(pi x) sin(pi y) sin(pi z)."""
    x = np.asarray(x)
    gy, gz = np.sin(PI * np.asarray(y)), np.sin(PI * np.asarray(z))
    ux = np.exp(x) * np.sin(PI * x)
    # -(e^x sin pi x)'' = e^x ((pi^2 - 1) sin pi x - 2 pi cos pi x); the y and
    # z factors each add pi^2 u.
    fx = np.exp(x) * ((3 * PI**2 - 1 + c) * np.sin(PI * x) - 2 * PI * np.cos(PI * x))
    return _outer3(ux, gy, gz), _outer3(fx, gy, gz)


def table1_dirichlet(x, y, z, alpha: float = 1.0):
    """u_D*(x) = sin(pi x) sin(2 pi y) sin(3 pi z) + (x - x^3)(y^2 - y^4)(1 - z^2)
    on [-1,1]^3 (Section 3.1) and f = alpha u - Lap u."""
    x, y, z = (np.asarray(t) for t in (x, y, z))
    s = _outer3(np.sin(PI * x), np.sin(2 * PI * y), np.sin(3 * PI * z))
    p, q, r = x - x**3, y**2 - y**4, 1 - z**2
    pdd, qdd, rdd = -6 * x, 2 - 12 * y**2, -2 * np.ones_like(z)
    u = s + _outer3(p, q, r)
    f = ((alpha + 14 * PI**2) * s + alpha * _outer3(p, q, r)
         - (_outer3(pdd, q, r) + _outer3(p, qdd, r) + _outer3(p, q, rdd)))
    return u, f


def random_rhs(nx: int, ny: int, nz: int, seed: int) -> np.ndarray:
    """i.i.d. N(0,1) nodal values (numpy PCG64, seeded)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal((nz, ny, nx))


@dataclass(frozen=True)
class Workload:
    """One solve workload: box [0,Lx]x[0,Ly]x[0,Lz], degree k, Ne elements per axis."""
    name: str
    k: int
    ne: tuple
    L: tuple
    c: float
    rhs: str  # "sine_123", "exp_sine" or "random"

    @property
    def n(self):
        return tuple(e * self.k - 1 for e in self.ne)

    @property
    def dofs(self) -> int:
        nx, ny, nz = self.n
        return nx * ny * nz


#: Q^2, 32 elements per axis on [0,1]^3, n = 63, -Lap u = f (single FP64 solve).
Q2_N63 = Workload("q2_n63_sine123", 2, (32, 32, 32), (1.0, 1.0, 1.0), 0.0, "sine_123")
#: Q^4, 250 elements per axis on [0,1]^3, n = 999 (~1.0e9 DoF), -Lap u + u = f.
Q4_N999 = Workload("q4_n999_expsine", 4, (250, 250, 250), (1.0, 1.0, 1.0), 1.0, "exp_sine")


def rhs_for(w: Workload, x, y, z, seed: int = 20231001):
    """(u_exact or None, f) for workload w at the given node coordinates."""
    if w.rhs == "sine_123":
        return sine_123(x, y, z)
    if w.rhs == "exp_sine":
        return exp_sine(x, y, z, w.c)
    if w.rhs == "random":
        return None, random_rhs(len(x), len(y), len(z), seed)
    raise ValueError(w.rhs)


def table1_neumann(x, y, z, alpha: float = 1.0):
    """u_N*(x) = cos(pi x) cos(2 pi y) cos(3 pi z) + (1-x^2)^3 (1-y^2)^2 (1-z^2)^4
    on [-1,1]^3 (Section 3.1, homogeneous Neumann data) and f = alpha u - Lap u."""
    x, y, z = (np.asarray(t) for t in (x, y, z))
    s = _outer3(np.cos(PI * x), np.cos(2 * PI * y), np.cos(3 * PI * z))
    p, q, r = (1 - x**2) ** 3, (1 - y**2) ** 2, (1 - z**2) ** 4
    pdd = (1 - x**2) * (30 * x**2 - 6)
    qdd = 12 * y**2 - 4
    rdd = (1 - z**2) ** 2 * (56 * z**2 - 8)
    u = s + _outer3(p, q, r)
    f = ((alpha + 14 * PI**2) * s + alpha * _outer3(p, q, r)
         - (_outer3(pdd, q, r) + _outer3(p, qdd, r) + _outer3(p, q, rdd)))
    return u, f


def harmonic_potential(x, y, z, amp: float = 100.0):
    """V(x) = amp |x - (0.5, 0.5, 0.5)|^2 at the nodes (the Schroedinger PCG
    workload on [0,1]^3); its mean over the unit cube is amp / 4."""
    x, y, z = (np.asarray(t) for t in (x, y, z))
    return amp * ((np.asarray(z)[:, None, None] - 0.5) ** 2 + (np.asarray(y)[None, :, None] - 0.5) ** 2
                  + (np.asarray(x)[None, None, :] - 0.5) ** 2)


def schrodinger_manufactured(x, y, z, amp: float = 100.0):
    """(u, V, f) with u = sin(pi x) sin(pi y) sin(pi z) and V = harmonic_potential:
    f = -Lap u + V u = (3 pi^2 + V) u."""
    u = _outer3(np.sin(PI * np.asarray(x)), np.sin(PI * np.asarray(y)), np.sin(PI * np.asarray(z)))
    V = harmonic_potential(x, y, z, amp)
    return u, V, (3 * PI**2 + V) * u


def batched_helmholtz(count: int = 64, seed: int = 20231001, sizes=(63, 127, 255, 383, 511), degrees=(2, 3, 4, 6)):
    """Problem list of the batched workload: for problem i a PCG64 generator
    seeded with seed + i draws k from `degrees`, each axis size uniformly from
    the entries of `sizes` with (n + 1) % k == 0, and c uniform in [0, 10].
    Boxes are [0,1]^3.  Returns dicts with n3, k, c and the seed of its f
    (i.i.d. N(0,1) from random_rhs)."""
    out = []
    for i in range(count):
        rng = np.random.Generator(np.random.PCG64(seed + i))
        k = int(rng.choice(np.asarray(degrees)))
        allowed = np.asarray([n for n in sizes if (n + 1) % k == 0])
        n3 = tuple(int(rng.choice(allowed)) for _ in range(3))
        c = float(rng.uniform(0.0, 10.0))
        out.append({"n3": n3, "k": k, "c": c, "seed": seed + 1000 + i})
    return out
