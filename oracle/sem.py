"""Plain FP64 CPU oracle of the Q^k spectral-element fast-diagonalisation solve.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Written from the paper
(arXiv 2310.00226), section by section:

* Section 2.1 / Eq. (4) (weak2D) and the 3D matrix form (Eq. 12, matvec3D):
  the Q^k SEM is continuous Q^k FEM with (k+1)-point Gauss-Lobatto (GLL)
  quadrature, so the 1D mass matrix M is diagonal and the 1D stiffness S is
  banded (one element's k+1 nodes couple).
* Section 2.2 (Eqs. 6-9): H = M^{-1} S = T Lambda T^{-1}, from the generalised
  eigenproblem S v = lambda M v.
* Section 2.3: robust form S1 = M^{-1/2} S M^{-1/2} = Q Lambda Q^T,
  T = M^{-1/2} Q, T^{-1} = Q^T M^{1/2}.
* Section 2.4, Eq. (13) (3D-Poisson) and the seven-step online solve that
  follows it: three mode products with T^{-1}, a pointwise division by
  lambda_x + lambda_y + lambda_z (+ alpha), three mode products with T.
* Appendix (LegendreD / SEGenerator1D): GLL nodes from Gauss-Jacobi(1,1) by the
  Golub-Welsch eigenvalue method, weights 2 / (N(N+1) P_N(r)^2), the
  barycentric differentiation matrix, element assembly ("glue") and the
  half-width scaling S/h, M*h.

Array convention: a 3D grid function is a numpy array of shape (nz, ny, nx),
C-contiguous, so that the flat index is i + nx*(j + ny*l) (x fastest), the
same order as the paper's vec(U) (Section 2.4).  Internally the paper's U(i,j,l)
is the transposed view ``G.T`` of shape (nx, ny, nz).

Homogeneous Dirichlet data are imposed by dropping the first and last global
node of each axis (Section 2.2 leaves the Dirichlet treatment to an earlier
paper); n = Ne*k - 1 interior nodes per axis.  This reading reproduces
the DoF counts and the l2 errors of Table 1 (pinned in the tests).
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp


# --------------------------------------------------------------------------
# 1D building blocks (Appendix: LegendreD)
# --------------------------------------------------------------------------

def legendre_p(N: int, x):
    """Standard Legendre polynomial P_N(x) (P_N(1) = 1) by the three-term
    recurrence (m+1) P_{m+1} = (2m+1) x P_m - m P_{m-1}."""
    x = np.asarray(x, dtype=np.float64)
    p_prev = np.ones_like(x)
    if N == 0:
        return p_prev
    p = x.copy()
    for m in range(1, N):
        p_prev, p = p, ((2 * m + 1) * x * p - m * p_prev) / (m + 1)
    return p


def _gauss_jacobi_nodes(alpha: float, beta: float, m: int) -> np.ndarray:
    """Nodes of the m-point Gauss-Jacobi rule for weight (1-x)^alpha (1+x)^beta.

    Golub-Welsch: the nodes are the eigenvalues of the symmetric tridiagonal
    matrix of the three-term recurrence of the Jacobi polynomials
    p_{j+1} = (x - a_j) p_j - b_j p_{j-1} (monic form), with
      a_j = (beta^2 - alpha^2) / ((2j+alpha+beta)(2j+alpha+beta+2)),
      b_j = 4 j (j+alpha)(j+beta)(j+alpha+beta)
            / ((2j+alpha+beta)^2 (2j+alpha+beta+1)(2j+alpha+beta-1)).
    The appendix's JacobiGQ does the same (Appendix, LegendreD).
    """
    if m == 0:
        return np.zeros(0)
    j = np.arange(m, dtype=np.float64)
    s = 2 * j + alpha + beta
    with np.errstate(divide="ignore", invalid="ignore"):
        a = (beta**2 - alpha**2) / (s * (s + 2))
    if abs(alpha + beta) < 1e-14:
        a[0] = (beta - alpha) / (alpha + beta + 2)
    jj = np.arange(1, m, dtype=np.float64)
    ss = 2 * jj + alpha + beta
    b = 4 * jj * (jj + alpha) * (jj + beta) * (jj + alpha + beta) / (ss**2 * (ss + 1) * (ss - 1))
    J = np.diag(a) + np.diag(np.sqrt(b), 1) + np.diag(np.sqrt(b), -1)
    return np.sort(np.linalg.eigvalsh(J))


def gll_nodes_weights(N: int):
    """(N+1)-point Gauss-Lobatto-Legendre nodes r (ascending) and weights w.

    Appendix (LegendreD / JacobiGL): the interior nodes are the N-1 Gauss nodes
    of Jacobi(1,1) (the zeros of P_N'), the end nodes are -1 and +1; the weights
    are w_i = 2 / (N (N+1) P_N(r_i)^2) (the appendix writes the same weight
    with the normalised Legendre polynomial).
    """
    if N < 1:
        raise ValueError("GLL rule needs N >= 1")
    interior = _gauss_jacobi_nodes(1.0, 1.0, N - 1)
    r = np.concatenate(([-1.0], interior, [1.0]))
    w = 2.0 / (N * (N + 1) * legendre_p(N, r) ** 2)
    return r, w


def diff_matrix(r: np.ndarray) -> np.ndarray:
    """Lagrange differentiation matrix D_ij = l_j'(r_i) on the nodes r.

    Appendix (LegendreD): barycentric form D_ij = (c_i / c_j) / (r_i - r_j) for
    i != j with c_i = prod_{m != i} (r_i - r_m); the diagonal is minus the
    off-diagonal row sum (derivative of a constant is zero).
    """
    n = len(r)
    diff = r[:, None] - r[None, :] + np.eye(n)
    c = np.prod(diff, axis=1)
    D = (c[:, None] / c[None, :]) / diff
    np.fill_diagonal(D, 0.0)
    np.fill_diagonal(D, -D.sum(axis=1))
    return D


# --------------------------------------------------------------------------
# 1D spectral-element matrices and eigenbasis (Sections 2.1-2.3, Appendix)
# --------------------------------------------------------------------------

@dataclass
class Sem1D:
    k: int              # polynomial degree
    Ne: int             # number of elements
    bc: str             # "dirichlet" or "neumann"
    x: np.ndarray       # node coordinates of the unknowns (length n)
    S: np.ndarray       # stiffness matrix (n x n, dense)
    M: np.ndarray       # diagonal of the lumped GLL mass matrix (length n)
    lam: np.ndarray     # eigenvalues of H = M^{-1} S, ascending
    Q: np.ndarray       # orthonormal eigenvectors of S1 = M^{-1/2} S M^{-1/2}
    T: np.ndarray       # T = M^{-1/2} Q   (columns: eigenvectors of H)
    Tinv: np.ndarray    # T^{-1} = Q^T M^{1/2}

    @property
    def n(self) -> int:
        return len(self.x)

    @property
    def H(self) -> np.ndarray:
        """H = M^{-1} S (Section 2.2, Eq. 6)."""
        return self.S / self.M[:, None]

    def H_sparse(self):
        return sp.csr_matrix(self.H)


def sem_1d(k: int, Ne: int, left: float, right: float, bc: str = "dirichlet") -> Sem1D:
    """Assemble S and M on [left, right] with Ne elements of degree k and
    diagonalise H = M^{-1} S robustly (Section 2.3).

    Element e spans [left + e*dx, left + (e+1)*dx]; its nodes are
    left + e*dx + h*(1 + r) with h = dx/2.  On the element,
    S_e = D^T diag(w) D / h and M_e = h * diag(w) (change of variables
    x = left + e*dx + h(1+r)).  Neighbouring elements share their end node
    (continuity, the appendix's "glue").  For Dirichlet data the first and
    last global nodes are removed.
    """
    if k < 1 or Ne < 1:
        raise ValueError("need k >= 1 and Ne >= 1")
    r, w = gll_nodes_weights(k)
    D = diff_matrix(r)
    dx = (right - left) / Ne
    h = dx / 2.0
    n_glob = Ne * k + 1
    xg = np.empty(n_glob)
    Sg = np.zeros((n_glob, n_glob))
    Mg = np.zeros(n_glob)
    S_loc = D.T @ np.diag(w) @ D
    for e in range(Ne):
        idx = e * k + np.arange(k + 1)
        xg[idx] = left + e * dx + h * (1.0 + r)
        Sg[np.ix_(idx, idx)] += S_loc / h
        Mg[idx] += w * h
    if bc == "dirichlet":
        keep = slice(1, n_glob - 1)
    elif bc == "neumann":
        keep = slice(0, n_glob)
    else:
        raise ValueError(bc)
    x = xg[keep].copy()
    S = Sg[keep, keep].copy()
    M = Mg[keep].copy()
    # Section 2.3: S1 = M^{-1/2} S M^{-1/2}, symmetric; eigen-decompose it.
    m_half_inv = 1.0 / np.sqrt(M)
    S1 = m_half_inv[:, None] * S * m_half_inv[None, :]
    S1 = 0.5 * (S1 + S1.T)
    lam, Q = np.linalg.eigh(S1)
    order = np.argsort(lam)
    lam, Q = lam[order], Q[:, order]
    # Sign convention (the sign of an eigenvector is free): make the largest
    # |entry| of each column positive.
    sgn = np.sign(Q[np.argmax(np.abs(Q), axis=0), np.arange(Q.shape[1])])
    sgn[sgn == 0] = 1.0
    Q = Q * sgn[None, :]
    T = m_half_inv[:, None] * Q
    Tinv = Q.T * np.sqrt(M)[None, :]
    return Sem1D(k=k, Ne=Ne, bc=bc, x=x, S=S, M=M, lam=lam, Q=Q, T=T, Tinv=Tinv)


# --------------------------------------------------------------------------
# 3D operators and the solve (Section 2.4)
# --------------------------------------------------------------------------

def mode_product(U: np.ndarray, A, axis: int) -> np.ndarray:
    """Contract axis `axis` of the 3D array U with matrix A:
    out[.., a, ..] = sum_i A[a, i] * U[.., i, ..]  (Eq. 11 / Eq. 12 of
    Section 2.4, one factor of the Kronecker product at a time).  A may be a
    dense array or a scipy sparse matrix."""
    Um = np.moveaxis(U, axis, 0)
    shp = Um.shape
    Y = A @ Um.reshape(shp[0], -1)
    Y = np.asarray(Y).reshape((A.shape[0],) + shp[1:])
    return np.moveaxis(Y, 0, axis)


def _paper_view(G: np.ndarray) -> np.ndarray:
    """(nz, ny, nx) x-fastest array -> the paper's U(i, j, l) view (nx, ny, nz)."""
    return G.T


def fast_solve(F: np.ndarray, sx: Sem1D, sy: Sem1D, sz: Sem1D, c: float) -> np.ndarray:
    """U = (T_z (x) T_y (x) T_x) [ (T^{-1} F) ./ (Lambda3D + c) ]  (Eq. 13 and
    the seven steps printed after it: z, y, x mode products with T^{-1}, the
    entrywise division, z, y, x mode products with T).

    F and the result are (nz, ny, nx) arrays (x fastest); F holds nodal values
    of the right-hand side of c u + (H_x (+) H_y (+) H_z) u = f.
    """
    U = _paper_view(np.asarray(F, dtype=np.float64))
    U = mode_product(U, sz.Tinv, 2)
    U = mode_product(U, sy.Tinv, 1)
    U = mode_product(U, sx.Tinv, 0)
    lam3d = sx.lam[:, None, None] + sy.lam[None, :, None] + sz.lam[None, None, :] + c
    U = U / lam3d
    U = mode_product(U, sz.T, 2)
    U = mode_product(U, sy.T, 1)
    U = mode_product(U, sx.T, 0)
    return np.ascontiguousarray(U.T)


def fast_solve_x_line(fx, fy, fz, sx: Sem1D, sy: Sem1D, sz: Sem1D, c: float, j: int, l: int) -> np.ndarray:
    """Nodal values u[l, j, :] of ``fast_solve`` for a rank-one right-hand side
    F[l, j, i] = fz[l] fy[j] fx[i], computed one x-line at a time so that it
    can be evaluated on grids far too large for the whole field.

    Eq. 13 for a separable F: T^{-1} acts on each factor alone
    (xh = T_x^{-1} fx, ...), the division by lambda_x,a + lambda_y,b +
    lambda_z,g + c couples the three spectral indices, and the backward
    products give
      u[l, j, i] = sum_a T_x[i, a] xh_a W_a,
      W_a = sum_{b, g} T_y[j, b] yh_b T_z[l, g] zh_g
                       / (lambda_x,a + lambda_y,b + lambda_z,g + c).
    Cost n_y n_z per spectral x-index: n^3 for the line."""
    xh = sx.Tinv @ np.asarray(fx, dtype=np.float64)
    yh = sy.Tinv @ np.asarray(fy, dtype=np.float64)
    zh = sz.Tinv @ np.asarray(fz, dtype=np.float64)
    P = (sz.T[l, :] * zh)[:, None] * (sy.T[j, :] * yh)[None, :]   # (g, b)
    lam_zy = sz.lam[:, None] + sy.lam[None, :] + c
    W = np.array([np.sum(P / (lam_zy + la)) for la in sx.lam])
    return sx.T @ (xh * W)


def apply_h(Ug: np.ndarray, sx: Sem1D, sy: Sem1D, sz: Sem1D, c: float) -> np.ndarray:
    """(c I + I(x)I(x)H_x + I(x)H_y(x)I + H_z(x)I(x)I) vec(U)  (Eq. 12 with
    H = M^{-1} S; the alpha term of Eq. 1 added as c).  Uses sparse H."""
    U = _paper_view(np.asarray(Ug, dtype=np.float64))
    out = c * U
    out = out + mode_product(U, sx.H_sparse(), 0)
    out = out + mode_product(U, sy.H_sparse(), 1)
    out = out + mode_product(U, sz.H_sparse(), 2)
    return np.ascontiguousarray(out.T)


def apply_weak(Ug: np.ndarray, sx: Sem1D, sy: Sem1D, sz: Sem1D, c: float) -> np.ndarray:
    """Weak-form operator A u = (c M(x)M(x)M + M(x)M(x)S_x + M(x)S_y(x)M +
    S_z(x)M(x)M) u  (Eq. 12, left-hand side, plus the alpha mass term of
    Eq. 2).  Dense 1D factors, used on small and medium grids."""
    U = _paper_view(np.asarray(Ug, dtype=np.float64))
    Mx, My, Mz = (sp.diags(s.M) for s in (sx, sy, sz))
    MU = mode_product(mode_product(mode_product(U, Mx, 0), My, 1), Mz, 2)
    out = c * MU
    out = out + mode_product(mode_product(mode_product(U, sp.csr_matrix(sx.S), 0), My, 1), Mz, 2)
    out = out + mode_product(mode_product(mode_product(U, Mx, 0), sp.csr_matrix(sy.S), 1), Mz, 2)
    out = out + mode_product(mode_product(mode_product(U, Mx, 0), My, 1), sp.csr_matrix(sz.S), 2)
    return np.ascontiguousarray(out.T)


def apply_mass(Ug: np.ndarray, sx: Sem1D, sy: Sem1D, sz: Sem1D) -> np.ndarray:
    """(M_z (x) M_y (x) M_x) vec(F): the right-hand side of Eq. 12."""
    return Ug * (sz.M[:, None, None] * sy.M[None, :, None] * sx.M[None, None, :])


def refined_solve(F: np.ndarray, sx: Sem1D, sy: Sem1D, sz: Sem1D, c: float, sweeps: int = 1) -> np.ndarray:
    """Fast solve followed by `sweeps` FP64 iterative-refinement sweeps:
    r = f - (c + H_x (+) H_y (+) H_z) u ;  u <- u + fast_solve(r).

    The paper's method is a direct solve; a bare FP64 fast solve is accurate to
    roughly n * 1e-14 against the exact discrete solution.  One FP64 sweep
    brings it to rounding level, which makes it a sharp reference."""
    u = fast_solve(F, sx, sy, sz, c)
    for _ in range(sweeps):
        r = F - apply_h(u, sx, sy, sz, c)
        u = u + fast_solve(r, sx, sy, sz, c)
    return u


def dense_solve(F: np.ndarray, sx: Sem1D, sy: Sem1D, sz: Sem1D, c: float) -> np.ndarray:
    """Plain definition of the discrete solution on tiny grids: assemble the
    weak-form matrix of Eq. 12 (plus c times the mass) with Kronecker products
    and solve A u = (M(x)M(x)M) f by dense LU.  vec() is x fastest, so the x
    factor is the right-most Kronecker factor (Eq. 11)."""
    Mx, My, Mz = (np.diag(s.M) for s in (sx, sy, sz))
    A = (c * np.kron(Mz, np.kron(My, Mx))
         + np.kron(Mz, np.kron(My, sx.S))
         + np.kron(Mz, np.kron(sy.S, Mx))
         + np.kron(sz.S, np.kron(My, Mx)))
    b = np.kron(Mz, np.kron(My, Mx)) @ np.asarray(F, dtype=np.float64).reshape(-1)
    u = np.linalg.solve(A, b)
    return u.reshape(F.shape)


def l2_error_table1(err: np.ndarray, Ne: int) -> float:
    """The "l2 error" of Table 1: sqrt(sum of squared nodal errors) / Ne^{3/2}.
    The paper does not define it; this reading reproduces its printed values
    (see the Table 1 pin)."""
    return float(np.sqrt(np.sum(np.asarray(err) ** 2)) / Ne**1.5)


# --------------------------------------------------------------------------
# Schroedinger-type problem (Section 3.3, Eq. 15): alpha u - Lap u + V(x) u = f
# --------------------------------------------------------------------------

def weak_matrix(sx: Sem1D, sy: Sem1D, sz: Sem1D, diag_weight=None):
    """Sparse weak-form matrix S(+)S(+)S + M3 diag(w) (Eq. 12 with the lumped
    GLL quadrature of a variable zeroth-order coefficient w at the nodes;
    x-fastest Kronecker order).  diag_weight: (nz, ny, nx) array or scalar."""
    Sx, Sy, Sz = (sp.csr_matrix(s.S) for s in (sx, sy, sz))
    Mx, My, Mz = (sp.diags(s.M) for s in (sx, sy, sz))
    K = (sp.kron(Mz, sp.kron(My, Sx)) + sp.kron(Mz, sp.kron(Sy, Mx)) + sp.kron(Sz, sp.kron(My, Mx)))
    if diag_weight is not None:
        M3 = (sz.M[:, None, None] * sy.M[None, :, None] * sx.M[None, None, :]).reshape(-1)
        w = np.broadcast_to(np.asarray(diag_weight, dtype=np.float64), (sz.n, sy.n, sx.n)).reshape(-1)
        K = K + sp.diags(M3 * w)
    return K.tocsc()


def schrodinger_solve(F: np.ndarray, V: np.ndarray, sx: Sem1D, sy: Sem1D, sz: Sem1D) -> np.ndarray:
    """Plain definition of the discrete solution of -Lap u + V u = f (SEM with
    lumped GLL quadrature, homogeneous Dirichlet data): solve
    (S(+)S(+)S + M3 diag(V)) u = M3 f by a sparse direct factorisation.  The
    paper solves it by PCG preconditioned with the fast solver of
    (alpha + beta/2) - Lap (Section 3.3); the discrete solution is the same."""
    import scipy.sparse.linalg as spla
    K = weak_matrix(sx, sy, sz, V)
    b = apply_mass(F, sx, sy, sz).reshape(-1)
    return spla.spsolve(K, b).reshape(F.shape)


# --------------------------------------------------------------------------
# Cahn-Hilliard BDF2 step (Section 3.5, Eqs. 17-20)
# --------------------------------------------------------------------------

def assembled_h3(sx: Sem1D, sy: Sem1D, sz: Sem1D) -> np.ndarray:
    """Dense H3 = I(x)I(x)H_x + I(x)H_y(x)I + H_z(x)I(x)I (x fastest): the
    discrete -Lap in H form (Eq. 12)."""
    Ix, Iy, Iz = (np.eye(s.n) for s in (sx, sy, sz))
    return np.kron(Iz, np.kron(Iy, sx.H)) + np.kron(Iz, np.kron(sy.H, Ix)) + np.kron(sz.H, np.kron(Iy, Ix))


def bdf2_history(phi_n: np.ndarray, phi_nm1: np.ndarray):
    """History terms of the BDF2 step (Eq. 19): with a = 3/2, the time
    derivative (a phi_{n+1} - phi_hat)/dt has phi_hat = 2 phi_n - phi_{n-1}/2,
    and the nonlinear term is taken at the second-order extrapolation
    phi_bar = 2 phi_n - phi_{n-1}.  Returns (phi_hat, phi_bar)."""
    return 2.0 * phi_n - 0.5 * phi_nm1, 2.0 * phi_n - phi_nm1


def ch_explicit_term(phi_bar: np.ndarray, eps: float, S: float) -> np.ndarray:
    """g = (F'(phi_bar) - S phi_bar) / eps with F'(phi) = phi^3 - phi (the
    derivative of F(phi) = (phi^2 - 1)^2 / 4, Section 3.5): the part of the
    chemical potential treated explicitly, minus the stabilisation's explicit
    half."""
    return (phi_bar**3 - phi_bar - S * phi_bar) / eps


def ch_step(phi_n: np.ndarray, phi_nm1: np.ndarray, sx: Sem1D, sy: Sem1D, sz: Sem1D,
            eps: float, m: float, dt: float, S: float = 0.0) -> np.ndarray:
    """One BDF2 step of the Cahn-Hilliard system (Eq. 19, with the chemical
    potential eliminated as in Eq. 20), on small grids, by a dense solve.

    phi_t = m Lap mu, mu = -eps Lap phi + F'(phi)/eps, F'(phi) = phi^3 - phi;
    BDF2 with a = 3/2, phi_hat = 2 phi_n - phi_{n-1}/2, extrapolated
    phi_bar = 2 phi_n - phi_{n-1} in the nonlinear term.  The stabilisation
    the paper borrows (Section 3.5.2, formula not printed) is read as
    mu_{n+1} += (S/eps)(phi_{n+1} - phi_bar); S = 0 is the paper's scheme.
    With -Lap -> H3 (homogeneous Dirichlet data for phi and Lap phi):
      (a + dt m (eps H3^2 + (S/eps) H3)) phi_{n+1}
          = phi_hat - dt m H3 g,   g = (F'(phi_bar) - S phi_bar) / eps.
    """
    H3 = assembled_h3(sx, sy, sz)
    a = 1.5
    phi_hat, phi_bar = bdf2_history(phi_n, phi_nm1)
    g = ch_explicit_term(phi_bar, eps, S)
    P = a * np.eye(H3.shape[0]) + dt * m * (eps * H3 @ H3 + (S / eps) * H3)
    rhs = phi_hat.reshape(-1) - dt * m * (H3 @ g.reshape(-1))
    return np.linalg.solve(P, rhs).reshape(phi_n.shape)
