"""FP64 oracle of the interpolated PSF Hessian and its image-domain CGNR (App. D).

TEST INFRASTRUCTURE ONLY (callers: tests/, smoke(), bench.py's CPU legs).

App. D samples the Hessian H = L^T L with a comb of point scatterers: the
PSF image L^T L comb holds, around each comb node, one localised column of H.
Because neighbouring PSFs look alike (local translation invariance), a column
at a point between the nodes is estimated by interpolating the node columns,
each taken relative to its own node, with the weights of Eq. (trilinear)
(bilinear in 2D). The interpolated operator is applied on the fly, and the
deconvolved image solves H^H H dm = H^H m_rtm by CGNR from dm = 0, which gives
the minimum-norm least-squares solution (the interpolated H is singular).

Definitions (the readings where App. D is silent are marked *):

  * nodes along an axis of length n: s//2 + k s < n, k = 0, 1, ... (the comb
    of the PSF probe, spacing s);
  * node patch (*): P_k(a) = Q(node_k + a) for |a_z|, |a_x| <= half, Q = 0
    outside the image; half defaults to (s - 1) // 2, the widest window that
    stays clear of the neighbouring nodes' windows. For s = 5 this is the
    5 x 5 window of the 30 x 30 example of App. D (5 band groups of 5 bands);
  * corners of a coordinate c (*): between the first and the last node,
    k0 = (c - node_0) // s, k1 = k0 + 1 and the weight w = (c - node_k0) / s,
    as in Eq. (trilinear); before the first or after the last node both
    corners are that node and w = 0 (constant extrapolation);
  * column at point c: H(c + a, c) = sum over the 4 corners (k0|k1 along z,
    k0|k1 along x) of the product of the two 1D weights ((1 - w) for k0, w
    for k1) times P_corner(a); entries with c + a outside the image are
    dropped;
  * two parameters: block (i, j) (output plane i, input plane j, 0 = Vp,
    1 = Ip) takes Q = plane i of the PSF of the comb in parameter j;
  * parameter mask (*): the operator is P H P, P keeping the planes in the
    mask (1 = Vp, 2 = Ip, 3 = both); the CG data are P m_rtm.

The columns are formed literally (interpolated patch times the input value,
spread over the window); numpy only vectorises the loop over pixels.

3D images ([2, nz, ny, nx]) use Eq. (trilinear) as printed: the eight
corners of the node cell around the voxel, weights (1 - w1 or w1) (1 - w2
or w2) (1 - w3 or w3) from the same per-axis rule, windows of (2 half + 1)^3.
"""
from __future__ import annotations

import numpy as np

from . import cgls
from .deblur import nodes


def default_half(s: int) -> int:
    """Half width of the node windows when none is given: (s - 1) // 2."""
    return (s - 1) // 2


def corners_1d(c: int, n: int, s: int) -> tuple[int, int, float]:
    """(k0, k1, w) of coordinate c on an axis of length n, node spacing s."""
    zk = nodes(n, s)
    if c <= zk[0]:
        return 0, 0, 0.0
    if c >= zk[-1]:
        k = len(zk) - 1
        return k, k, 0.0
    k0 = (c - zk[0]) // s
    return int(k0), int(k0) + 1, (c - zk[k0]) / s


def axis_corners(n: int, s: int):
    """corners_1d for every coordinate of an axis, as three arrays."""
    t = [corners_1d(c, n, s) for c in range(n)]
    return (np.array([a for a, _, _ in t]), np.array([b for _, b, _ in t]),
            np.array([w for _, _, w in t], np.float64))


def patches(Q: np.ndarray, s: int, half: int) -> np.ndarray:
    """Node patches [nkz, nkx, 2 half + 1, 2 half + 1] of one PSF plane Q."""
    nz, nx = Q.shape
    zk, xk = nodes(nz, s), nodes(nx, s)
    L = 2 * half + 1
    P = np.zeros((len(zk), len(xk), L, L))
    for i, z in enumerate(zk):
        for j, x in enumerate(xk):
            for a in range(-half, half + 1):
                for b in range(-half, half + 1):
                    if 0 <= z + a < nz and 0 <= x + b < nx:
                        P[i, j, a + half, b + half] = Q[z + a, x + b]
    return P


def column(P: np.ndarray, s: int, nz: int, nx: int, cz: int, cx: int) -> np.ndarray:
    """Interpolated column patch H(c + a, c), a in the window (Eq. trilinear, 2D)."""
    kz0, kz1, wz = corners_1d(cz, nz, s)
    kx0, kx1, wx = corners_1d(cx, nx, s)
    return ((1 - wz) * (1 - wx) * P[kz0, kx0] + (1 - wz) * wx * P[kz0, kx1]
            + wz * (1 - wx) * P[kz1, kx0] + wz * wx * P[kz1, kx1])


def patches3(Q: np.ndarray, s: int, half: int) -> np.ndarray:
    """Node patches [nkz, nky, nkx, L, L, L] (L = 2 half + 1) of one 3D PSF plane Q."""
    nz, ny, nx = Q.shape
    zk, yk, xk = nodes(nz, s), nodes(ny, s), nodes(nx, s)
    L = 2 * half + 1
    P = np.zeros((len(zk), len(yk), len(xk), L, L, L))
    for i, z in enumerate(zk):
        for j, y in enumerate(yk):
            for k, x in enumerate(xk):
                for a in range(-half, half + 1):
                    for b in range(-half, half + 1):
                        for c in range(-half, half + 1):
                            if 0 <= z + a < nz and 0 <= y + b < ny and 0 <= x + c < nx:
                                P[i, j, k, a + half, b + half, c + half] = Q[z + a, y + b, x + c]
    return P


def column3(P: np.ndarray, s: int, shape, cz: int, cy: int, cx: int) -> np.ndarray:
    """Interpolated column patch H(c + a, c) of a 3D image: Eq. (trilinear), the
    eight corners (z0|z1, y0|y1, x0|x1) with the products of the 1D weights."""
    nz, ny, nx = shape
    kz0, kz1, w3 = corners_1d(cz, nz, s)
    ky0, ky1, w2 = corners_1d(cy, ny, s)
    kx0, kx1, w1 = corners_1d(cx, nx, s)
    return ((1 - w1) * (1 - w2) * (1 - w3) * P[kz0, ky0, kx0] + w1 * (1 - w2) * (1 - w3) * P[kz0, ky0, kx1]
            + (1 - w1) * w2 * (1 - w3) * P[kz0, ky1, kx0] + w1 * w2 * (1 - w3) * P[kz0, ky1, kx1]
            + (1 - w1) * (1 - w2) * w3 * P[kz1, ky0, kx0] + w1 * (1 - w2) * w3 * P[kz1, ky0, kx1]
            + (1 - w1) * w2 * w3 * P[kz1, ky1, kx0] + w1 * w2 * w3 * P[kz1, ky1, kx1])


def _planes(mask: int) -> list[int]:
    return [q for q in (0, 1) if mask & (1 << q)]


def block_patches(psf_vp, psf_ip, s: int, half: int, mask: int = 3) -> dict:
    """Patches of the blocks (i, j) with i, j in the mask; psf_vp / psf_ip are
    the [2, nz, nx] PSF images of the combs in Vp / Ip."""
    src = (psf_vp, psf_ip)
    out = {}
    for j in _planes(mask):
        if src[j] is None:
            raise ValueError(f"the PSF of parameter {j} is needed for mask {mask}")
        for i in _planes(mask):
            plane = np.asarray(src[j], np.float64)[i]
            out[(i, j)] = patches(plane, s, half) if plane.ndim == 2 else patches3(plane, s, half)
    return out


def _column_fields(P: np.ndarray, s: int, nz: int, nx: int, half: int):
    """For every window offset a, the field C_a[c] = H(c + a, c) over all c."""
    kz0, kz1, wz = axis_corners(nz, s)
    kx0, kx1, wx = axis_corners(nx, s)
    Z0, X0 = np.meshgrid(kz0, kx0, indexing="ij")
    Z1, X1 = np.meshgrid(kz1, kx1, indexing="ij")
    WZ, WX = np.meshgrid(wz, wx, indexing="ij")
    for a in range(-half, half + 1):
        for b in range(-half, half + 1):
            p = P[:, :, a + half, b + half]
            C = ((1 - WZ) * (1 - WX) * p[Z0, X0] + (1 - WZ) * WX * p[Z0, X1]
                 + WZ * (1 - WX) * p[Z1, X0] + WZ * WX * p[Z1, X1])
            yield a, b, C


def _shift(g: np.ndarray, a: int, b: int) -> np.ndarray:
    """g(p - (a, b)), zero where p - (a, b) leaves the image."""
    out = np.zeros_like(g)
    nz, nx = g.shape
    zs, ze = max(0, a), min(nz, nz + a)
    xs, xe = max(0, b), min(nx, nx + b)
    if zs < ze and xs < xe:
        out[zs:ze, xs:xe] = g[zs - a:ze - a, xs - b:xe - b]
    return out


def _column_fields3(P: np.ndarray, s: int, shape, half: int):
    """3D: for every window offset a, the field C_a[c] = H(c + a, c) over all c."""
    nz, ny, nx = shape
    kz0, kz1, w3 = axis_corners(nz, s)
    ky0, ky1, w2 = axis_corners(ny, s)
    kx0, kx1, w1 = axis_corners(nx, s)
    I = np.ix_
    for a in range(-half, half + 1):
        for b in range(-half, half + 1):
            for c in range(-half, half + 1):
                p = P[:, :, :, a + half, b + half, c + half]
                C = np.zeros(shape)
                for kz, wz in ((kz0, 1 - w3), (kz1, w3)):
                    for ky, wy in ((ky0, 1 - w2), (ky1, w2)):
                        for kx, wx in ((kx0, 1 - w1), (kx1, w1)):
                            C += (wz[:, None, None] * wy[None, :, None] * wx[None, None, :]) * p[I(kz, ky, kx)]
                yield (a, b, c), C


def _shift_nd(g: np.ndarray, off) -> np.ndarray:
    """g(p - off), zero where p - off leaves the array."""
    out = np.zeros_like(g)
    src, dst = [], []
    for n, a in zip(g.shape, off):
        s0, e0 = max(0, a), min(n, n + a)
        if s0 >= e0:
            return out
        dst.append(slice(s0, e0))
        src.append(slice(s0 - a, e0 - a))
    out[tuple(dst)] = g[tuple(src)]
    return out


def _apply3(blocks: dict, s: int, half: int, x: np.ndarray, transpose: bool) -> np.ndarray:
    y = np.zeros_like(x)
    for (i, j), P in blocks.items():
        for off, C in _column_fields3(P, s, x.shape[1:], half):
            if not transpose:
                y[i] += _shift_nd(C * x[j], off)
            else:
                y[j] += C * _shift_nd(x[i], tuple(-o for o in off))
    return y


def apply(blocks: dict, s: int, half: int, x: np.ndarray, transpose: bool = False) -> np.ndarray:
    """y = P H P x (or P H^T P x): x, y [2, nz, nx] or [2, nz, ny, nx]; `blocks`
    from block_patches."""
    x = np.asarray(x, np.float64)
    if x.ndim == 4:
        return _apply3(blocks, s, half, x, transpose)
    nz, nx = x.shape[1:]
    y = np.zeros_like(x)
    for (i, j), P in blocks.items():
        for a, b, C in _column_fields(P, s, nz, nx, half):
            if not transpose:
                # column c of block (i, j) times x_j[c], placed at c + (a, b)
                y[i] += _shift(C * x[j], a, b)
            else:
                # <column c of block (i, j), y_i>, read at c + (a, b)
                y[j] += C * _shift(x[i], -a, -b)
    return y


def apply_at(blocks: dict, s: int, half: int, x: np.ndarray, plane: int, rz: int, rx: int,
             transpose: bool = False) -> float:
    """One output value of apply(), column by column (for large images)."""
    x = np.asarray(x, np.float64)
    nz, nx = x.shape[1:]
    acc = 0.0
    for (i, j), P in blocks.items():
        if (j if transpose else i) != plane:
            continue
        if transpose:
            col = column(P, s, nz, nx, rz, rx)
            for a in range(-half, half + 1):
                for b in range(-half, half + 1):
                    if 0 <= rz + a < nz and 0 <= rx + b < nx:
                        acc += col[a + half, b + half] * x[i, rz + a, rx + b]
        else:
            for a in range(-half, half + 1):
                for b in range(-half, half + 1):
                    cz, cx = rz - a, rx - b
                    if 0 <= cz < nz and 0 <= cx < nx and x[j, cz, cx] != 0.0:
                        acc += column(P, s, nz, nx, cz, cx)[a + half, b + half] * x[j, cz, cx]
    return acc


def _explicit3(blocks: dict, s: int, half: int, shape) -> np.ndarray:
    nz, ny, nx = shape
    nv = nz * ny * nx
    H = np.zeros((2 * nv, 2 * nv))
    r = range(-half, half + 1)
    for (i, j), P in blocks.items():
        for cz in range(nz):
            for cy in range(ny):
                for cx in range(nx):
                    col = column3(P, s, shape, cz, cy, cx)
                    for a in r:
                        for b in r:
                            for c in r:
                                z, y, x = cz + a, cy + b, cx + c
                                if 0 <= z < nz and 0 <= y < ny and 0 <= x < nx:
                                    H[i * nv + (z * ny + y) * nx + x, j * nv + (cz * ny + cy) * nx + cx] = \
                                        col[a + half, b + half, c + half]
    return H


def explicit(blocks: dict, s: int, half: int, shape) -> np.ndarray:
    """Dense P H P written entry by entry from column() / column3() (tiny
    images only); rows and columns index [plane][z][(y)][x]."""
    if len(shape) == 3:
        return _explicit3(blocks, s, half, shape)
    nz, nx = shape
    n = 2 * nz * nx
    H = np.zeros((n, n))
    for (i, j), P in blocks.items():
        for cz in range(nz):
            for cx in range(nx):
                col = column(P, s, nz, nx, cz, cx)
                for a in range(-half, half + 1):
                    for b in range(-half, half + 1):
                        if 0 <= cz + a < nz and 0 <= cx + b < nx:
                            H[(i * nz + cz + a) * nx + cx + b, (j * nz + cz) * nx + cx] = col[a + half, b + half]
    return H


def cgnr(blocks: dict, s: int, half: int, m_rtm: np.ndarray, niter: int, mask: int = 3):
    """CGNR on H^H H dm = H^H P m_rtm from dm = 0; returns (dm, normalised
    misfits ||P m_rtm - H dm_k|| / ||P m_rtm||, k = 0..niter)."""
    d = np.asarray(m_rtm, np.float64).copy()
    for q in (0, 1):
        if not mask & (1 << q):
            d[q] = 0.0
    return cgls(lambda v: apply(blocks, s, half, v), lambda v: apply(blocks, s, half, v, True),
                d, np.zeros_like(d), niter, param_mask=mask)
