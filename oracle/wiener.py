"""FP64 oracle of the nonstationary Wiener filter (App. E, Fourier form).

TEST INFRASTRUCTURE ONLY (callers: tests/, smoke(), bench.py's CPU legs).

App. E treats the Hessian as locally translation invariant: within a local
block it is circulant, diagonalised by the Fourier matrix F, so H = F^H Lam F
and dm = F^H Lam^-1 F m_rtm (Eq. sol). Lam^-1 is estimated per wavenumber i
from the reference image m' and its remigration m'' = H m' by the
Tikhonov-regularised least squares
    min sum_i |[F m']_i - Lam_i^-1 [F m'']_i|^2 + eps |Lam_i^-1|^2,
solved by the Wiener ratio Lam_i^-1 = conj([F m'']_i) [F m']_i /
(conj([F m'']_i) [F m'']_i + eps), with m' = m_rtm. The block results are
blended with valence weights, dm = sum_k w_k dm_k / sum_k w_k.

Readings where App. E is silent (shared with the CUDA path):
  * blocks: one per comb node (z_k, x_k) = (s/2 + i s, s/2 + j s) inside the
    image, the 2s x 2s pixels z_k - s .. z_k + s - 1, x_k - s .. x_k + s - 1
    (zero outside the image), so neighbouring blocks overlap by half;
  * eps is relative: eps_k = eps * mean_i |[F m'']_i|^2 of the block (a block
    whose m'' is zero gets Lam^-1 = 0);
  * F is the unnormalised 2D DFT of the block (numpy.fft.fft2) and F^H F = I
    is kept by the 1/(2s)^2 of the inverse (numpy.fft.ifft2); the block's
    result is the real part;
  * valence: the bilinear hat w_k(p) = max(0, 1 - |z - z_k|/s)
    max(0, 1 - |x - x_k|/s), as for the space-domain filters; pixels that no
    node covers get 0;
  * every parameter plane is filtered on its own.
"""
from __future__ import annotations

import numpy as np

from .deblur import nodes


def block(g: np.ndarray, zc: int, xc: int, s: int) -> np.ndarray:
    """The 2s x 2s block of g around (zc, xc), zero outside the image."""
    nz, nx = g.shape
    out = np.zeros((2 * s, 2 * s))
    z0, x0 = zc - s, xc - s
    zs, ze = max(0, z0), min(nz, z0 + 2 * s)
    xs, xe = max(0, x0), min(nx, x0 + 2 * s)
    if zs < ze and xs < xe:
        out[zs - z0:ze - z0, xs - x0:xe - x0] = g[zs:ze, xs:xe]
    return out


def inverse_eigenvalues(m_ref_blk: np.ndarray, m_rem_blk: np.ndarray, eps: float) -> np.ndarray:
    """Lam^-1 of one block: the Wiener ratio of App. E with eps_k = eps * mean |F m''|^2."""
    A = np.fft.fft2(m_rem_blk)
    B = np.fft.fft2(m_ref_blk)
    power = np.abs(A) ** 2
    if not np.any(power > 0.0):
        return np.zeros_like(A)
    eps_k = eps * float(np.mean(power))
    return np.conj(A) * B / (power + eps_k)


def block_filter(m_rtm_blk: np.ndarray, m_rem_blk: np.ndarray, eps: float) -> np.ndarray:
    """dm_k = Re F^H Lam^-1 F m_rtm on one block (m' = m_rtm)."""
    lam_inv = inverse_eigenvalues(m_rtm_blk, m_rem_blk, eps)
    return np.real(np.fft.ifft2(lam_inv * np.fft.fft2(m_rtm_blk)))


def wiener_plane(m_rtm: np.ndarray, m_remig: np.ndarray, s: int, eps: float) -> np.ndarray:
    """One parameter plane: block filters blended with the bilinear valence."""
    nz, nx = m_rtm.shape
    num = np.zeros((nz, nx))
    den = np.zeros((nz, nx))
    for z in nodes(nz, s):
        for x in nodes(nx, s):
            dmk = block_filter(block(m_rtm, z, x, s), block(m_remig, z, x, s), eps)
            # the hat's support (|z - z_k| < s, |x - x_k| < s) lies inside the
            # block, so the sums run over the block's pixels in the image
            z0, x0 = z - s, x - s
            zs, ze = max(0, z0), min(nz, z0 + 2 * s)
            xs, xe = max(0, x0), min(nx, x0 + 2 * s)
            wz = np.maximum(0.0, 1.0 - np.abs(np.arange(zs, ze) - z) / s)[:, None]
            wx = np.maximum(0.0, 1.0 - np.abs(np.arange(xs, xe) - x) / s)[None, :]
            num[zs:ze, xs:xe] += wz * wx * dmk[zs - z0:ze - z0, xs - x0:xe - x0]
            den[zs:ze, xs:xe] += wz * wx
    return np.where(den > 0.0, num / np.where(den > 0.0, den, 1.0), 0.0)


def wiener(m_rtm: np.ndarray, m_remig: np.ndarray, spacing: int, eps: float = 1e-3) -> np.ndarray:
    """Nonstationary Wiener deblurring of a [2, nz, nx] image pair."""
    m_rtm = np.asarray(m_rtm, np.float64)
    m_remig = np.asarray(m_remig, np.float64)
    return np.stack([wiener_plane(m_rtm[q], m_remig[q], spacing, eps) for q in range(m_rtm.shape[0])])
