"""FP64 oracle of the nonstationary deblurring filters (App. E).

TEST INFRASTRUCTURE ONLY (callers: tests/, smoke(), bench.py's CPU legs).

App. E connects the reference image m' and the remigrated image
m'' = L^T L m' = H m' through a convolution with the inverse of a locally
translation-invariant Hessian: f * m'' ~= m'. The filter is estimated per
local block by regularised least squares, applied to the migrated image
(delta m = f * m_rtm, Eq. sol with m' = m_rtm), and the block results are
blended with valence weights, delta m = sum_k w_k delta m_k / sum_k w_k.

The paper estimates each block's filter in the wavenumber domain; this build
estimates it in space as a flen x flen (11 x 11) FIR filter, the same
regularised least-squares problem restricted to short filters:

  * nodes: (z_k, x_k) = (s/2 + i s, s/2 + j s) inside the image (the PSF comb
    of App. D, spacing s);
  * window W_k: the pixels within s of the node in z and in x, clipped to the
    image;
  * filter: f_k = argmin_f sum_{p in W_k} ((f * m'')(p) - m'(p))^2
                          + eps_k ||f||^2,
    (f * g)(p) = sum_{|a|,|b| <= h} f[a, b] g(p - (a, b)), h = flen // 2,
    g = 0 outside the image, eps_k = eps * trace(A^T A) / flen^2;
    solved through the FP64 normal equations (A^T A + eps_k I) f = A^T m'
    (a window whose A^T A is zero gets the zero filter);
  * blending: w_k(p) = max(0, 1 - |z - z_k| / s) * max(0, 1 - |x - x_k| / s)
    (bilinear valence), delta m(p) = sum_k w_k(p) (f_k * m_rtm)(p) /
    sum_k w_k(p) (0 where no node covers p);
  * every parameter plane is filtered on its own (no cross-parameter filter).

The matrix A and the convolutions are written out as plain loops over the
window and the filter taps; numpy's Cholesky factorisation solves the
normal equations.
"""
from __future__ import annotations

import numpy as np


def nodes(n: int, s: int) -> np.ndarray:
    """Comb node coordinates s/2, s/2 + s, ... below n along one axis."""
    return np.arange(s // 2, n, s)


def window(n: int, c: int, s: int) -> tuple[int, int]:
    """Half-open index range of the window around node c along one axis."""
    return max(0, c - s), min(n, c + s + 1)


def shifted(g: np.ndarray, a: int, b: int) -> np.ndarray:
    """g(p - (a, b)) on the image grid, zero where p - (a, b) leaves it."""
    out = np.zeros_like(g)
    nz, nx = g.shape
    zs, ze = max(0, a), min(nz, nz + a)
    xs, xe = max(0, b), min(nx, nx + b)
    out[zs:ze, xs:xe] = g[zs - a:ze - a, xs - b:xe - b]
    return out


def taps(flen: int) -> list[tuple[int, int]]:
    """Filter taps (a, b), a and b in [-h, h], row-major in a."""
    h = flen // 2
    return [(a, b) for a in range(-h, h + 1) for b in range(-h, h + 1)]


def design_matrix(m2: np.ndarray, zr, xr, flen: int) -> np.ndarray:
    """A[p, (a, b)] = m''(p - (a, b)) for p in the window (rows row-major)."""
    cols = [shifted(m2, a, b)[zr[0]:zr[1], xr[0]:xr[1]].ravel() for a, b in taps(flen)]
    return np.stack(cols, axis=1)


def window_filter(m1: np.ndarray, m2: np.ndarray, zr, xr, flen: int, eps: float) -> np.ndarray:
    """Regularised least-squares filter of one window, [flen, flen]."""
    A = design_matrix(m2, zr, xr, flen)
    y = m1[zr[0]:zr[1], xr[0]:xr[1]].ravel()
    N = A.T @ A
    tr = float(np.trace(N))
    if tr == 0.0:
        return np.zeros((flen, flen))
    N = N + eps * tr / (flen * flen) * np.eye(flen * flen)
    Lc = np.linalg.cholesky(N)
    f = np.linalg.solve(Lc.T, np.linalg.solve(Lc, A.T @ y))
    return f.reshape(flen, flen)


def convolve(f: np.ndarray, g: np.ndarray) -> np.ndarray:
    """(f * g)(p) = sum_{a, b} f[a, b] g(p - (a, b)) with g zero outside."""
    h = f.shape[0] // 2
    out = np.zeros_like(g)
    for a, b in taps(f.shape[0]):
        out += f[a + h, b + h] * shifted(g, a, b)
    return out


def filters(m_rtm: np.ndarray, m_remig: np.ndarray, spacing: int, flen: int = 11,
            eps: float = 1e-3) -> np.ndarray:
    """Filters of every node of one parameter plane, [nkz, nkx, flen, flen]."""
    nz, nx = m_rtm.shape
    zk, xk = nodes(nz, spacing), nodes(nx, spacing)
    out = np.zeros((len(zk), len(xk), flen, flen))
    for i, z in enumerate(zk):
        for j, x in enumerate(xk):
            out[i, j] = window_filter(m_rtm, m_remig, window(nz, z, spacing), window(nx, x, spacing),
                                      flen, eps)
    return out


def blend(m_rtm: np.ndarray, F: np.ndarray, spacing: int) -> np.ndarray:
    """delta m = sum_k w_k (f_k * m_rtm) / sum_k w_k with bilinear valence."""
    nz, nx = m_rtm.shape
    zk, xk = nodes(nz, spacing), nodes(nx, spacing)
    num = np.zeros((nz, nx))
    den = np.zeros((nz, nx))
    zz = np.arange(nz)[:, None].astype(np.float64)
    xx = np.arange(nx)[None, :].astype(np.float64)
    for i, z in enumerate(zk):
        wz = np.maximum(0.0, 1.0 - np.abs(zz - z) / spacing)
        for j, x in enumerate(xk):
            w = wz * np.maximum(0.0, 1.0 - np.abs(xx - x) / spacing)
            num += w * convolve(F[i, j], m_rtm)
            den += w
    return np.where(den > 0, num / np.where(den > 0, den, 1.0), 0.0)


def deblur(m_rtm: np.ndarray, m_remig: np.ndarray, spacing: int, flen: int = 11,
           eps: float = 1e-3):
    """Deblurred image and filters for [nparam, nz, nx] inputs, each plane on
    its own. Returns (delta m [nparam, nz, nx], filters [nparam, nkz, nkx, flen, flen])."""
    m_rtm = np.asarray(m_rtm, np.float64)
    m_remig = np.asarray(m_remig, np.float64)
    out = np.zeros_like(m_rtm)
    Fs = []
    for q in range(m_rtm.shape[0]):
        F = filters(m_rtm[q], m_remig[q], spacing, flen, eps)
        out[q] = blend(m_rtm[q], F, spacing)
        Fs.append(F)
    return out, np.stack(Fs)
