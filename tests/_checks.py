"""Residual-based checks shared by the GPU tests: rows of the weak-form
operator S(+)S(+)S + M3 diag(shift) applied to a block of a device array
(oracle matrices), and the componentwise and normwise backward errors of a
solution on sampled x-lines.  Test infrastructure; no GPU compute."""

import numpy as np


def _lines(ny, nz, count, seed):
    """Sampled (j, l) line indexes: the four corners of the (y, z) plane, the
    centre, and `count` seeded random ones."""
    rng = np.random.Generator(np.random.PCG64(seed))
    fixed = [(0, 0), (ny - 1, nz - 1), (0, nz - 1), (ny - 1, 0), (ny // 2, nz // 3)]
    rand = [(int(rng.integers(ny)), int(rng.integers(nz))) for _ in range(count)]
    return fixed + rand


def _block(t, l, j, r):
    """t[l-r : l+r+1, j-r : j+r+1, :] clipped to the grid, as numpy, with its origin."""
    nz, ny = t.shape[0], t.shape[1]
    l0, l1 = max(0, l - r), min(nz, l + r + 1)
    j0, j1 = max(0, j - r), min(ny, j + r + 1)
    return t[l0:l1, j0:j1, :].cpu().numpy(), l0, j0


def _kron_lines(B, l0, j0, pairs, Ax, Ay, Az, Mx, My, Mz):
    """Rows (l, j) of (Mz (x) My (x) Ax + Mz (x) Ay (x) Mx + Az (x) My (x) Mx) B,
    with B = G[l0:, j0:, :] a block of the grid function G that holds the bands
    of rows l and j (the 1D factors are banded with half-width k)."""
    out = []
    for (l, j) in pairs:
        bl, bj = l - l0, j - j0
        line = B[bl, bj]
        v = Mz[l] * My[j] * (Ax @ line)
        v = v + Mz[l] * Mx * (Ay[j, j0:j0 + B.shape[1]] @ B[bl])
        v = v + My[j] * Mx * (Az[l, l0:l0 + B.shape[0]] @ B[:, bj])
        out.append(v)
    return out


def _norm_inf_weak(sx, sy, sz, c):
    """||S(+)S(+)S + c M3||_inf: the largest row sum of |A|, one z-plane at a time."""
    rx, ry, rz = (np.abs(s.S).sum(1) for s in (sx, sy, sz))
    plane = rx[None, :] * sy.M[:, None] + sx.M[None, :] * ry[:, None] + c * sx.M[None, :] * sy.M[:, None]
    mm = sx.M[None, :] * sy.M[:, None]
    return float(max((sz.M[l] * plane + rz[l] * mm).max() for l in range(sz.n)))


def _normwise_backward_error(u_dev, f_dev, sx, sy, sz, c, pairs, k, a_inf, b_inf):
    """max over the sampled lines of |b - A u| / (||A|| ||u|| + ||b||)."""
    rmax = 0.0
    for (j, l) in pairs:
        B, l0, j0 = _block(u_dev, l, j, k)
        m3 = sz.M[l] * sy.M[j] * sx.M
        Au = _kron_lines(B, l0, j0, [(l, j)], sx.S, sy.S, sz.S, sx.M, sy.M, sz.M)[0]
        r = m3 * f_dev[l, j].cpu().numpy() - Au - m3 * c * B[l - l0, j - j0]
        rmax = max(rmax, float(np.abs(r).max()))
    return rmax / (a_inf * float(u_dev.abs().max()) + b_inf)


def _backward_error(u_dev, f_dev, sx, sy, sz, shift, pairs, k):
    """max over the sampled lines of |b - A u| / (|A| |u| + |b|) for the weak
    form A = S(+)S(+)S + M3 diag(shift), b = M3 f (Eq. 12 with the alpha term)."""
    eta = 0.0
    for (j, l) in pairs:
        B, l0, j0 = _block(u_dev, l, j, k)
        f = f_dev[l, j].cpu().numpy()
        s_line = shift if np.isscalar(shift) else shift[l, j].cpu().numpy()
        m3 = sz.M[l] * sy.M[j] * sx.M
        Au = _kron_lines(B, l0, j0, [(l, j)], sx.S, sy.S, sz.S, sx.M, sy.M, sz.M)[0]
        aAu = _kron_lines(np.abs(B), l0, j0, [(l, j)], np.abs(sx.S), np.abs(sy.S), np.abs(sz.S),
                          sx.M, sy.M, sz.M)[0]
        line = B[l - l0, j - j0]
        r = m3 * f - Au - m3 * s_line * line
        den = aAu + m3 * np.abs(s_line * line) + m3 * np.abs(f)
        eta = max(eta, float(np.max(np.abs(r) / den)))
    return eta
