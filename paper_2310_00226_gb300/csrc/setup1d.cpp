// Host FP64 construction of the 1D spectral-element data of one axis:
// GLL nodes and weights, differentiation matrix, assembled stiffness S and
// lumped mass M with homogeneous Dirichlet rows removed, and the robust
// eigenbasis T = M^{-1/2} Q, T^{-1} = Q^T M^{1/2} of H = M^{-1} S
// (Section 2.3 of arXiv 2310.00226; the setup the paper's appendix performs
// in its 1D generator).  Everything here runs once per plan, off the solve.
#include "sem3d_internal.h"

#include <algorithm>
#include <cmath>
#include <limits>
#include <stdexcept>
#include <vector>

namespace sem3d {

namespace {

// Legendre P_N(x) and P_{N-1}(x) by the three-term recurrence.
void legendre_pair(int N, double x, double* pN, double* pNm1) {
  double p0 = 1.0, p1 = x;
  if (N == 0) { *pN = 1.0; *pNm1 = 0.0; return; }
  for (int m = 1; m < N; ++m) {
    double p2 = ((2.0 * m + 1.0) * x * p1 - m * p0) / (m + 1.0);
    p0 = p1;
    p1 = p2;
  }
  *pN = p1;
  *pNm1 = p0;
}

}  // namespace

// GLL nodes: +-1 and the zeros of P_N'.  Newton's method on
// q(x) = (1 - x^2) P_N'(x) = N (P_{N-1}(x) - x P_N(x)), using the Legendre
// equation q'(x) = -N (N+1) P_N(x):  x <- x + (P_{N-1} - x P_N) / ((N+1) P_N).
// Start: Chebyshev-Gauss-Lobatto points -cos(pi j / N).
// Weights w_j = 2 / (N (N+1) P_N(x_j)^2).
void gll_rule(int N, std::vector<double>& r, std::vector<double>& w) {
  r.assign(N + 1, 0.0);
  w.assign(N + 1, 0.0);
  r[0] = -1.0;
  r[N] = 1.0;
  for (int j = 1; j < N; ++j) {
    double x = -std::cos(M_PI * j / N);
    for (int it = 0; it < 100; ++it) {
      double pN, pNm1;
      legendre_pair(N, x, &pN, &pNm1);
      double dx = (pNm1 - x * pN) / ((N + 1.0) * pN);
      x += dx;
      if (std::fabs(dx) < 1e-17) break;
    }
    r[j] = x;
  }
  // exact symmetry about 0
  for (int j = 0; j <= N / 2; ++j) {
    double s = 0.5 * (r[N - j] - r[j]);
    r[j] = -s;
    r[N - j] = s;
  }
  if (N % 2 == 0) r[N / 2] = 0.0;
  for (int j = 0; j <= N; ++j) {
    double pN, pNm1;
    legendre_pair(N, r[j], &pN, &pNm1);
    w[j] = 2.0 / (N * (N + 1.0) * pN * pN);
  }
}

// Closed-form GLL differentiation matrix D_ij = l_j'(r_i):
//   i != j : P_N(r_i) / (P_N(r_j) (r_i - r_j))
//   D_00 = -N(N+1)/4, D_NN = N(N+1)/4, other diagonal entries 0.
void gll_diff(int N, const std::vector<double>& r, std::vector<double>& D) {
  const int n = N + 1;
  std::vector<double> p(n);
  for (int i = 0; i < n; ++i) {
    double pN, pNm1;
    legendre_pair(N, r[i], &pN, &pNm1);
    p[i] = pN;
  }
  D.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      if (i != j) D[(size_t)i * n + j] = p[i] / (p[j] * (r[i] - r[j]));
  D[0] = -N * (N + 1.0) / 4.0;
  D[(size_t)n * n - 1] = N * (N + 1.0) / 4.0;
}

namespace {

// Symmetric eigen-decomposition A = V diag(d) V^T of a dense n x n matrix
// (row-major, overwritten).  Householder reduction to tridiagonal form with
// the reflectors accumulated into V, then implicit QR steps with Wilkinson
// shifts on the tridiagonal matrix, rotating V along.  Eigenvalues
// are returned ascending with matching columns of V (V row-major: V[i*n+j] is
// component i of eigenvector j).
void sym_eig(int n, std::vector<double>& A, std::vector<double>& d, std::vector<double>& V) {
  V.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  std::vector<double> e(n, 0.0), v(n), p(n), wv(n);
  if (n == 1) { d.assign(1, A[0]); return; }
  d.assign(n, 0.0);
  auto a = [&](int i, int j) -> double& { return A[(size_t)i * n + j]; };
  // --- Householder tridiagonalisation: column k below the subdiagonal.
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;  // length of x = A[k+1.., k]
    double norm = 0.0;
    for (int t = 0; t < m; ++t) norm += a(k + 1 + t, k) * a(k + 1 + t, k);
    norm = std::sqrt(norm);
    if (norm == 0.0) continue;
    double x0 = a(k + 1, k);
    double alpha = x0 > 0 ? -norm : norm;
    for (int t = 0; t < m; ++t) v[t] = a(k + 1 + t, k);
    v[0] -= alpha;
    double vn = 0.0;
    for (int t = 0; t < m; ++t) vn += v[t] * v[t];
    vn = std::sqrt(vn);
    if (vn == 0.0) continue;
    for (int t = 0; t < m; ++t) v[t] /= vn;
    // p = A22 v, K = v^T p, w = p - K v ; A22 -= 2 (v w^T + w v^T)
#pragma omp parallel for schedule(static) if (m >= 256)
    for (int r = 0; r < m; ++r) {
      double s = 0.0;
      const double* row = &A[(size_t)(k + 1 + r) * n + (k + 1)];
      for (int t = 0; t < m; ++t) s += row[t] * v[t];
      p[r] = s;
    }
    double K = 0.0;
    for (int t = 0; t < m; ++t) K += v[t] * p[t];
    for (int t = 0; t < m; ++t) wv[t] = p[t] - K * v[t];
#pragma omp parallel for schedule(static) if (m >= 256)
    for (int r = 0; r < m; ++r) {
      double* row = &A[(size_t)(k + 1 + r) * n + (k + 1)];
      const double vr = 2.0 * v[r], wr = 2.0 * wv[r];
      for (int t = 0; t < m; ++t) row[t] -= vr * wv[t] + wr * v[t];
    }
    a(k + 1, k) = alpha;
    a(k, k + 1) = alpha;
    for (int t = 1; t < m; ++t) { a(k + 1 + t, k) = 0.0; a(k, k + 1 + t) = 0.0; }
    // V <- V (I - 2 v v^T) on columns k+1..n-1
#pragma omp parallel for schedule(static) if (n >= 256)
    for (int r = 0; r < n; ++r) {
      double* row = &V[(size_t)r * n + (k + 1)];
      double s = 0.0;
      for (int t = 0; t < m; ++t) s += row[t] * v[t];
      s *= 2.0;
      for (int t = 0; t < m; ++t) row[t] -= s * v[t];
    }
  }
  for (int i = 0; i < n; ++i) d[i] = a(i, i);
  for (int i = 0; i + 1 < n; ++i) e[i] = a(i + 1, i);
  // --- implicit symmetric tridiagonal QR with Wilkinson shifts (the
  // bulge-chasing step of Golub & Van Loan, "Matrix Computations", Sec. 8.3).
  // Diagonal d[0..n), off-diagonal e[i] between rows i and i+1.  Each step on
  // the unreduced block [lo, hi] records its Givens rotations (cs[], sn[]) and
  // then applies them to every row of V (independent rows, run in parallel).
  std::vector<double> cs(n), sn(n);
  const double eps = std::numeric_limits<double>::epsilon();
  int hi = n - 1, guard = 0;
  while (hi > 0) {
    if (std::fabs(e[hi - 1]) <= eps * (std::fabs(d[hi - 1]) + std::fabs(d[hi]))) {
      e[hi - 1] = 0.0;
      --hi;
      guard = 0;
      continue;
    }
    if (++guard > 200) throw std::runtime_error("symmetric eigen-solver did not converge");
    int lo = hi - 1;
    while (lo > 0 && std::fabs(e[lo - 1]) > eps * (std::fabs(d[lo - 1]) + std::fabs(d[lo]))) --lo;
    // Wilkinson shift from the trailing 2x2 block of [lo, hi].
    const double half = 0.5 * (d[hi - 1] - d[hi]);
    const double bb = e[hi - 1];
    const double mu = d[hi] - bb * bb / (half + (half >= 0 ? 1.0 : -1.0) * std::hypot(half, bb));
    double x = d[lo] - mu, z = e[lo], bulge = 0.0;
    for (int kk = lo; kk < hi; ++kk) {
      const double rr = std::hypot(x, z);
      const double c = rr == 0.0 ? 1.0 : x / rr, s = rr == 0.0 ? 0.0 : z / rr;
      if (kk > lo) e[kk - 1] = rr;  // (kk, kk-1) entry; the bulge is gone
      const double ak = d[kk], ak1 = d[kk + 1], bk = e[kk];
      d[kk] = c * c * ak + 2.0 * c * s * bk + s * s * ak1;
      d[kk + 1] = s * s * ak - 2.0 * c * s * bk + c * c * ak1;
      e[kk] = c * s * (ak1 - ak) + (c * c - s * s) * bk;
      if (kk + 1 < hi) {  // rotating columns kk, kk+1 of row kk+2 makes a bulge
        bulge = s * e[kk + 1];
        e[kk + 1] = c * e[kk + 1];
      }
      cs[kk] = c;
      sn[kk] = s;
      x = e[kk];
      z = bulge;
    }
#pragma omp parallel for schedule(static) if (n >= 256)
    for (int r = 0; r < n; ++r) {
      double* row = &V[(size_t)r * n];
      for (int kk = lo; kk < hi; ++kk) {
        const double vk = row[kk], vk1 = row[kk + 1];
        row[kk] = cs[kk] * vk + sn[kk] * vk1;
        row[kk + 1] = -sn[kk] * vk + cs[kk] * vk1;
      }
    }
  }
  // --- sort ascending (selection sort on indices, swap columns of V)
  for (int i = 0; i < n - 1; ++i) {
    int kmin = i;
    for (int j = i + 1; j < n; ++j)
      if (d[j] < d[kmin]) kmin = j;
    if (kmin != i) {
      std::swap(d[i], d[kmin]);
      for (int r = 0; r < n; ++r) std::swap(V[(size_t)r * n + i], V[(size_t)r * n + kmin]);
    }
  }
}

}  // namespace

// Build the axis data of degree k on [0, L]: n interior nodes (Dirichlet,
// bc = 0) or all n nodes (Neumann, bc = 1).
Axis1D build_axis(int n, int k, double L, int bc) {
  if (k < 1 || n < 1) throw std::invalid_argument("need n >= 1, k >= 1");
  if (bc == 0 && (n + 1) % k != 0) throw std::invalid_argument("Dirichlet: need (n+1) % k == 0");
  if (bc == 1 && (n < k + 1 || (n - 1) % k != 0)) throw std::invalid_argument("Neumann: need (n-1) % k == 0, n > k");
  if (bc != 0 && bc != 1) throw std::invalid_argument("unknown boundary condition");
  Axis1D ax;
  ax.n = n;
  ax.k = k;
  ax.bc = bc;
  ax.Ne = bc == 0 ? (n + 1) / k : (n - 1) / k;
  ax.L = L;
  const int offset = bc == 0 ? 1 : 0;  // unknown index = global node - offset
  std::vector<double> r, w, D;
  gll_rule(k, r, w);
  gll_diff(k, r, D);
  const int nl = k + 1;
  // Local stiffness on the reference element: S_loc = D^T diag(w) D.
  std::vector<double> Sloc((size_t)nl * nl, 0.0);
  for (int p = 0; p < nl; ++p)
    for (int q = 0; q < nl; ++q) {
      double s = 0.0;
      for (int m = 0; m < nl; ++m) s += D[(size_t)m * nl + p] * w[m] * D[(size_t)m * nl + q];
      Sloc[(size_t)p * nl + q] = s;
    }
  const double dx = L / ax.Ne, h = 0.5 * dx;
  // Global node g = e*k + q; unknown index = g - offset (Dirichlet: node 0 and
  // node Ne*k carry the boundary data and are dropped; Neumann: all kept).
  ax.x.assign(n, 0.0);
  ax.M.assign(n, 0.0);
  ax.S.assign((size_t)n * n, 0.0);
  for (int e = 0; e < ax.Ne; ++e) {
    for (int p = 0; p < nl; ++p) {
      const int gp = e * k + p - offset;
      if (gp < 0 || gp >= n) continue;
      ax.x[gp] = e * dx + h * (1.0 + r[p]);
      ax.M[gp] += h * w[p];
      for (int q = 0; q < nl; ++q) {
        const int gq = e * k + q - offset;
        if (gq < 0 || gq >= n) continue;
        ax.S[(size_t)gp * n + gq] += Sloc[(size_t)p * nl + q] / h;
      }
    }
  }
  // Robust eigenproblem (Section 2.3): S1 = M^{-1/2} S M^{-1/2}, symmetrised.
  std::vector<double> S1((size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double a = ax.S[(size_t)i * n + j] / std::sqrt(ax.M[i] * ax.M[j]);
      double b = ax.S[(size_t)j * n + i] / std::sqrt(ax.M[i] * ax.M[j]);
      S1[(size_t)i * n + j] = 0.5 * (a + b);
    }
  std::vector<double> Q;
  sym_eig(n, S1, ax.lam, Q);
  // Sign convention: largest |entry| of each eigenvector positive.
  for (int j = 0; j < n; ++j) {
    int imax = 0;
    for (int i = 1; i < n; ++i)
      if (std::fabs(Q[(size_t)i * n + j]) > std::fabs(Q[(size_t)imax * n + j])) imax = i;
    if (Q[(size_t)imax * n + j] < 0)
      for (int i = 0; i < n; ++i) Q[(size_t)i * n + j] = -Q[(size_t)i * n + j];
  }
  // T[i][j] = Q[i][j] / sqrt(M_i);  Tinv[j][i] = Q[i][j] * sqrt(M_i).
  ax.T.assign((size_t)n * n, 0.0);
  ax.Tinv.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) {
    const double sm = std::sqrt(ax.M[i]);
    for (int j = 0; j < n; ++j) {
      ax.T[(size_t)i * n + j] = Q[(size_t)i * n + j] / sm;
      ax.Tinv[(size_t)j * n + i] = Q[(size_t)i * n + j] * sm;
    }
  }
  // Band of H = M^{-1} S: row i couples columns [lo_i, hi_i] (one or two
  // elements), stored as H[i][i+d] for d in [-k, k].
  const int bw = 2 * k + 1;
  ax.Hband.assign((size_t)n * bw, 0.0);
  ax.band_lo.assign(n, 0);
  ax.band_hi.assign(n, 0);
  for (int i = 0; i < n; ++i) {
    int lo = n, hi = -1;
    for (int d = -k; d <= k; ++d) {
      const int j = i + d;
      if (j < 0 || j >= n) continue;
      const double v = ax.S[(size_t)i * n + j];
      if (v != 0.0) { lo = std::min(lo, j); hi = std::max(hi, j); }
      ax.Hband[(size_t)i * bw + (d + k)] = v / ax.M[i];
    }
    ax.band_lo[i] = lo;
    ax.band_hi[i] = hi;
  }
  // Per-local-index rows of H on the uniform mesh, summed in the same order as
  // the assembly above (left element first at a shared vertex), so that they
  // equal the assembled rows bit for bit.
  ax.Hq.assign((size_t)k * bw, 0.0);
  for (int q = 0; q < k; ++q) {
    const double Mq = (q == 0) ? (0.0 + h * w[k]) + h * w[0] : 0.0 + h * w[q];
    for (int d = -k; d <= k; ++d) {
      double sv = 0.0;
      if (q == 0) {
        if (d <= 0) sv += Sloc[(size_t)k * nl + (k + d)] / h;
        if (d >= 0) sv += Sloc[(size_t)0 * nl + d] / h;
      } else if (d >= -q && d <= k - q) {
        sv += Sloc[(size_t)q * nl + (q + d)] / h;
      }
      ax.Hq[(size_t)q * bw + (d + k)] = sv / Mq;
    }
  }
  return ax;
}

}  // namespace sem3d
