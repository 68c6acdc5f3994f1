"""Pins of the oracle's interpolated PSF Hessian and image-domain CGNR (App. D).

* a PSF that is the same at every node makes H a plain 2D convolution (and
  H^T a correlation): scipy's convolve2d / correlate2d;
* at a node the interpolated column is that node's PSF window, exactly;
* node PSFs that vary affinely over the nodes interpolate exactly (bilinear
  weights of Eq. trilinear), and beyond the last node they are constant;
* the 30 x 30 example of App. D (scatterers every 5 points) has 5 band groups
  of 5 bands (golden fixture, from the figure caption);
* the vectorised operator equals the dense matrix built column by column from
  the definition, and its transpose mode equals that matrix's transpose;
* CGNR from zero reaches the minimum-norm least-squares solution (numpy's
  pseudo-inverse) on an H whose two parameter columns coincide;
* with zero cross-parameter PSFs the two-parameter operator decouples."""
import json
import os

import numpy as np
import pytest

import lsrtm_inputs as li
from oracle import psf_hessian as ph

HERE = os.path.dirname(os.path.abspath(__file__))


def _image_from_patches(nz, nx, s, half, patch_of_node):
    """PSF plane with patch_of_node(i, j) [2h+1, 2h+1] around node (i, j)."""
    Q = np.zeros((nz, nx))
    for i, z in enumerate(range(s // 2, nz, s)):
        for j, x in enumerate(range(s // 2, nx, s)):
            p = patch_of_node(i, j)
            for a in range(-half, half + 1):
                for b in range(-half, half + 1):
                    if 0 <= z + a < nz and 0 <= x + b < nx:
                        Q[z + a, x + b] = p[a + half, b + half]
    return Q


def test_stationary_psf_is_a_convolution():
    signal = pytest.importorskip("scipy.signal")
    nz, nx, s, half = 40, 48, 8, 3    # every node window inside the image
    rng = np.random.default_rng(0)
    p = rng.standard_normal((2 * half + 1, 2 * half + 1))
    Q = _image_from_patches(nz, nx, s, half, lambda i, j: p)
    psf = np.stack([Q, np.zeros_like(Q)])
    bl = ph.block_patches(psf, None, s, half, mask=1)
    x = np.zeros((2, nz, nx))
    x[0] = rng.standard_normal((nz, nx))
    y = ph.apply(bl, s, half, x)
    assert np.allclose(y[0], signal.convolve2d(x[0], p, mode="same"), rtol=0, atol=1e-12)
    assert np.all(y[1] == 0)
    yt = ph.apply(bl, s, half, x, transpose=True)
    assert np.allclose(yt[0], signal.correlate2d(x[0], p, mode="same"), rtol=0, atol=1e-12)


def test_columns_at_nodes_are_the_node_psfs():
    nz, nx, s = 41, 53, 10
    half = ph.default_half(s)
    psf_vp, psf_ip = li.psf_images(nz, nx, s, seed=2)
    bl = ph.block_patches(psf_vp, psf_ip, s, half)
    for z in range(s // 2, nz, s):
        for x in range(s // 2, nx, s):
            e = np.zeros((2, nz, nx))
            e[1, z, x] = 1.0
            col = ph.apply(bl, s, half, e)
            z0, z1 = max(0, z - half), min(nz, z + half + 1)
            x0, x1 = max(0, x - half), min(nx, x + half + 1)
            for q in range(2):
                win = np.zeros((nz, nx))
                win[z0:z1, x0:x1] = psf_ip[q, z0:z1, x0:x1]
                assert np.array_equal(col[q], win)


def test_affine_node_psfs_interpolate_exactly():
    nz, nx, s, half = 48, 59, 8, 3
    zk, xk = np.arange(s // 2, nz, s), np.arange(s // 2, nx, s)
    assert zk[-1] + half < nz and xk[-1] + half < nx   # every node window inside the image
    q = np.random.default_rng(1).standard_normal((2 * half + 1, 2 * half + 1))
    f = lambda z, x: 0.7 + 0.013 * z - 0.021 * x
    Q = _image_from_patches(nz, nx, s, half, lambda i, j: f(zk[i], xk[j]) * q)
    bl = ph.block_patches(np.stack([Q, Q]), None, s, half, mask=1)
    P = bl[(0, 0)]
    for cz in range(nz):
        for cx in range(nx):
            col = ph.column(P, s, nz, nx, cz, cx)
            ez = min(max(cz, zk[0]), zk[-1])   # constant beyond the end nodes
            ex = min(max(cx, xk[0]), xk[-1])
            assert np.allclose(col, f(ez, ex) * q, rtol=0, atol=1e-13)
    # the sampled operator reproduces the same columns
    cz, cx = 21, 30
    e = np.zeros((2, nz, nx))
    e[0, cz, cx] = 1.0
    y = ph.apply(bl, s, half, e)
    assert np.allclose(y[0, cz - half:cz + half + 1, cx - half:cx + half + 1], f(cz, cx) * q, atol=1e-13)


def test_banded_structure_of_the_30x30_example():
    with open(os.path.join(HERE, "golden", "psf_hessian_banded_30x30.json")) as fh:
        g = json.load(fh)
    nz, nx, s = g["nz"], g["nx"], g["spacing"]
    half = ph.default_half(s)
    psf_vp, _ = li.psf_images(nz, nx, s, seed=4)
    bl = ph.block_patches(psf_vp, None, s, half, mask=1)
    H = ph.explicit(bl, s, half, (nz, nx))[:nz * nx, :nz * nx]
    rows, cols = np.nonzero(H)
    offsets = np.unique(rows - cols)
    groups = np.unique(np.round(offsets / nx).astype(int))
    assert len(groups) == g["band_groups"]
    per = [np.sum(np.round(offsets / nx).astype(int) == k) for k in groups]
    assert per == [g["bands_per_group"]] * g["band_groups"]
    # each band lies within (2 half + 1) of its group's diagonal
    assert np.all(np.abs(offsets - np.round(offsets / nx) * nx) <= half)


@pytest.mark.parametrize("mask", [1, 2, 3])
def test_operator_equals_its_explicit_columns(mask):
    nz, nx, s = 13, 17, 6
    half = ph.default_half(s)
    psf_vp, psf_ip = li.psf_images(nz, nx, s, seed=5)
    bl = ph.block_patches(psf_vp, psf_ip, s, half, mask=mask)
    H = ph.explicit(bl, s, half, (nz, nx))
    rng = np.random.default_rng(6)
    x = rng.standard_normal((2, nz, nx))
    y = rng.standard_normal((2, nz, nx))
    keep = np.zeros((2, nz, nx))
    for qq in (0, 1):
        if mask & (1 << qq):
            keep[qq] = 1.0
    assert np.allclose(ph.apply(bl, s, half, x).ravel(), H @ (keep * x).ravel(), atol=1e-12)
    assert np.allclose(ph.apply(bl, s, half, y, transpose=True).ravel(), H.T @ (keep * y).ravel(), atol=1e-12)
    for plane, rz, rx in ((mask.bit_length() - 1, 0, 0), (mask.bit_length() - 1, 7, 16)):
        ref_f = (H @ (keep * x).ravel()).reshape(2, nz, nx)[plane, rz, rx]
        ref_t = (H.T @ (keep * y).ravel()).reshape(2, nz, nx)[plane, rz, rx]
        assert abs(ph.apply_at(bl, s, half, x, plane, rz, rx) - ref_f) < 1e-12
        assert abs(ph.apply_at(bl, s, half, y, plane, rz, rx, transpose=True) - ref_t) < 1e-12


def test_cgnr_reaches_the_minimum_norm_solution():
    nz, nx, s, half = 12, 12, 4, 1
    a, _ = li.psf_images(nz, nx, s, seed=3)
    bl = ph.block_patches(a, a.copy(), s, half)    # the Ip columns repeat the Vp columns
    H = ph.explicit(bl, s, half, (nz, nx))
    assert np.linalg.matrix_rank(H) == nz * nx
    d = np.random.default_rng(1).standard_normal((2, nz, nx))
    ref = np.linalg.pinv(H, rcond=1e-12) @ d.ravel()
    x, mis = ph.cgnr(bl, s, half, d, 400)
    assert np.linalg.norm(x.ravel() - ref) <= 1e-9 * np.linalg.norm(ref)
    assert np.array_equal(x[0], x[1])
    assert np.all(np.diff(mis) <= 1e-12) and mis[0] == 1.0


def test_two_parameters_without_cross_terms_decouple():
    nz, nx, s = 33, 41, 10
    half = ph.default_half(s)
    a, b = li.psf_images(nz, nx, s, seed=8)
    a[1] = 0.0
    b[0] = 0.0
    x = np.random.default_rng(2).standard_normal((2, nz, nx))
    both = ph.apply(ph.block_patches(a, b, s, half), s, half, x)
    vp = ph.apply(ph.block_patches(a, None, s, half, mask=1), s, half, x)
    ip = ph.apply(ph.block_patches(None, b, s, half, mask=2), s, half, x)
    assert np.allclose(both, vp + ip, rtol=0, atol=1e-13)
    with pytest.raises(ValueError):
        ph.block_patches(a, None, s, half, mask=3)


# ------------------------------------------------------------------ 3D


def _volume_from_patches(shape, s, half, patch_of_node):
    Q = np.zeros(shape)
    nz, ny, nx = shape
    for i, z in enumerate(range(s // 2, nz, s)):
        for j, y in enumerate(range(s // 2, ny, s)):
            for k, x in enumerate(range(s // 2, nx, s)):
                p = patch_of_node(i, j, k)
                Q[z - half:z + half + 1, y - half:y + half + 1, x - half:x + half + 1] = p
    return Q


def test_stationary_psf_is_a_convolution_3d():
    ndimage = pytest.importorskip("scipy.ndimage")
    shape, s, half = (20, 14, 26), 6, 2     # every node window inside the volume
    rng = np.random.default_rng(10)
    p = rng.standard_normal((2 * half + 1,) * 3)
    Q = _volume_from_patches(shape, s, half, lambda i, j, k: p)
    bl = ph.block_patches(np.stack([Q, 0 * Q]), None, s, half, mask=1)
    x = np.zeros((2,) + shape)
    x[0] = rng.standard_normal(shape)
    y = ph.apply(bl, s, half, x)
    assert np.allclose(y[0], ndimage.convolve(x[0], p, mode="constant"), rtol=0, atol=1e-12)
    yt = ph.apply(bl, s, half, x, transpose=True)
    assert np.allclose(yt[0], ndimage.correlate(x[0], p, mode="constant"), rtol=0, atol=1e-12)


def test_affine_node_psfs_interpolate_exactly_3d():
    shape, s, half = (20, 14, 26), 6, 2
    zk, yk, xk = (np.arange(s // 2, n, s) for n in shape)
    q = np.random.default_rng(11).standard_normal((2 * half + 1,) * 3)
    f = lambda z, y, x: 0.6 + 0.011 * z - 0.017 * y + 0.023 * x
    Q = _volume_from_patches(shape, s, half, lambda i, j, k: f(zk[i], yk[j], xk[k]) * q)
    P = ph.block_patches(np.stack([Q, Q]), None, s, half, mask=1)[(0, 0)]
    for cz in range(shape[0]):
        for cy in range(0, shape[1], 3):
            for cx in range(0, shape[2], 5):
                col = ph.column3(P, s, shape, cz, cy, cx)
                ez = min(max(cz, zk[0]), zk[-1])
                ey = min(max(cy, yk[0]), yk[-1])
                ex = min(max(cx, xk[0]), xk[-1])
                assert np.allclose(col, f(ez, ey, ex) * q, rtol=0, atol=1e-13)


def test_operator_equals_its_explicit_columns_3d():
    shape, s = (5, 6, 7), 3
    half = ph.default_half(s)
    pv, pi = li.psf_images3(*shape, s, seed=12)
    bl = ph.block_patches(pv, pi, s, half)
    H = ph.explicit(bl, s, half, shape)
    rng = np.random.default_rng(13)
    x = rng.standard_normal((2,) + shape)
    y = rng.standard_normal((2,) + shape)
    assert np.allclose(ph.apply(bl, s, half, x).ravel(), H @ x.ravel(), atol=1e-12)
    assert np.allclose(ph.apply(bl, s, half, y, transpose=True).ravel(), H.T @ y.ravel(), atol=1e-12)


def test_two_parameter_solution_follows_the_block_inverse():
    """The partitioned inverse behind the multiparameter inversion: with
    N = H^T H in 2 x 2 parameter blocks and b = H^T m, the two-parameter
    solution is the block inverse of N applied to b (Schur complement
    S = N11 - N12 N22^-1 N21; x2 = N22^-1 b2 - N22^-1 N21 x1), which the
    oracle's two-parameter CGNR reaches; its mono-parameter (Ip) CGNR reaches
    the solution of the Ip block alone (P H P), which the coupling term makes
    different."""
    nz, nx, s, half = 10, 12, 4, 1
    pv, pi = li.psf_images(nz, nx, s, seed=21)
    bl = ph.block_patches(pv, pi, s, half)
    H = ph.explicit(bl, s, half, (nz, nx))
    n = nz * nx
    N = H.T @ H
    N11, N12, N21, N22 = N[:n, :n], N[:n, n:], N[n:, :n], N[n:, n:]
    m = np.random.default_rng(22).standard_normal((2, nz, nx))
    b = H.T @ m.ravel()
    b1, b2 = b[:n], b[n:]
    N22i = np.linalg.inv(N22)
    S = N11 - N12 @ N22i @ N21
    x1 = np.linalg.solve(S, b1 - N12 @ N22i @ b2)
    x2 = N22i @ b2 - N22i @ N21 @ x1
    assert np.allclose(np.concatenate([x1, x2]), np.linalg.solve(N, b), rtol=0, atol=1e-8 * np.abs(x1).max())
    x, _ = ph.cgnr(bl, s, half, m, 600)
    assert np.allclose(x.ravel(), np.concatenate([x1, x2]), rtol=0, atol=1e-7 * np.abs(x1).max())
    # mono-parameter (Ip): the data are P m, the operator P H P
    bl2 = ph.block_patches(None, pi, s, half, mask=2)
    xm, _ = ph.cgnr(bl2, s, half, m, 600, mask=2)
    H22 = H[n:, n:]
    x2_mono = np.linalg.solve(H22.T @ H22, H22.T @ m[1].ravel())
    assert np.allclose(xm[1].ravel(), x2_mono, rtol=0, atol=1e-7 * np.abs(x2_mono).max())
    assert np.all(xm[0] == 0.0)
    # the paper's point: the two differ, by the coupling term
    assert not np.allclose(x2, x2_mono, atol=1e-3 * np.abs(x2).max())


def test_cgnr_reaches_the_minimum_norm_solution_3d():
    shape, s, half = (6, 6, 6), 3, 1
    a, _ = li.psf_images3(*shape, s, seed=14)
    bl = ph.block_patches(a, a.copy(), s, half)    # the Ip columns repeat the Vp columns
    H = ph.explicit(bl, s, half, shape)
    d = np.random.default_rng(15).standard_normal((2,) + shape)
    ref = np.linalg.pinv(H, rcond=1e-12) @ d.ravel()
    x, mis = ph.cgnr(bl, s, half, d, 800)     # cond(H) ~ 480 on its range: ~800 iterations in FP64
    assert np.linalg.norm(x.ravel() - ref) <= 1e-8 * np.linalg.norm(ref)
    assert np.array_equal(x[0], x[1])
