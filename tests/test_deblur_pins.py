"""Pins of the deblurring-filter oracle (App. E) against brute force, least
squares and cases whose filter is known in closed form."""
import numpy as np

from oracle import deblur as db


def _brute_design(m2, zr, xr, flen):
    h = flen // 2
    nz, nx = m2.shape
    rows = []
    for z in range(*zr):
        for x in range(*xr):
            row = []
            for a in range(-h, h + 1):
                for b in range(-h, h + 1):
                    zz, xx = z - a, x - b
                    row.append(m2[zz, xx] if 0 <= zz < nz and 0 <= xx < nx else 0.0)
            rows.append(row)
    return np.array(rows)


def test_filter_equals_regularised_lstsq():
    rng = np.random.default_rng(1)
    m1 = rng.standard_normal((23, 19))
    m2 = rng.standard_normal((23, 19))
    for zr, xr in (((0, 9), (3, 14)), ((10, 23), (0, 19)), ((5, 16), (8, 19))):
        A = _brute_design(m2, zr, xr, 5)
        y = m1[zr[0]:zr[1], xr[0]:xr[1]].ravel()
        eps = 1e-2 * np.trace(A.T @ A) / 25
        Aa = np.vstack([A, np.sqrt(eps) * np.eye(25)])
        ya = np.concatenate([y, np.zeros(25)])
        ref = np.linalg.lstsq(Aa, ya, rcond=None)[0].reshape(5, 5)
        got = db.window_filter(m1, m2, zr, xr, 5, 1e-2)
        assert np.abs(got - ref).max() < 1e-10 * np.abs(ref).max()


def test_convolution_brute_force():
    rng = np.random.default_rng(2)
    f = rng.standard_normal((5, 5))
    g = rng.standard_normal((9, 12))
    out = np.zeros_like(g)
    for z in range(9):
        for x in range(12):
            for a in range(-2, 3):
                for b in range(-2, 3):
                    if 0 <= z - a < 9 and 0 <= x - b < 12:
                        out[z, x] += f[a + 2, b + 2] * g[z - a, x - b]
    assert np.abs(db.convolve(f, g) - out).max() < 1e-12


def test_scaled_hessian_gives_scaled_image():
    """m'' = c m' makes f = delta / c exact in every window (eps = 0), so the
    blended image is m_rtm / c whatever the valence weights."""
    rng = np.random.default_rng(3)
    m = rng.standard_normal((2, 47, 61))
    out, F = db.deblur(m, 2.5 * m, spacing=10, flen=11, eps=0.0)
    delta = np.zeros((11, 11))
    delta[5, 5] = 1 / 2.5
    assert np.abs(F - delta).max() < 1e-9
    assert np.abs(out - m / 2.5).max() < 1e-9


def test_shifted_hessian_gives_opposite_shift():
    """m''(q) = m'(q - t) inside an interior window: f = delta at a = -t."""
    rng = np.random.default_rng(4)
    big = rng.standard_normal((60, 60))
    t = (1, -2)
    m1 = big[5:55, 5:55]
    m2 = big[5 - t[0]:55 - t[0], 5 - t[1]:55 - t[1]]
    f = db.window_filter(m1, m2, (15, 36), (12, 33), 11, 0.0)
    ref = np.zeros((11, 11))
    ref[5 - t[0], 5 - t[1]] = 1.0
    assert np.abs(f - ref).max() < 1e-9


def test_blur_is_inverted_inside_the_band():
    """A separable 3-tap blur h (response 0.7 + 0.3 cos w >= 0.4, so its
    inverse decays geometrically and an 11-tap filter nearly reaches it)
    applied to a white image: f * m'' reproduces m' to 1e-3 of the blur's own
    misfit, and f has the inverse's unit DC gain."""
    rng = np.random.default_rng(5)
    big = rng.standard_normal((90, 90))
    k = np.array([0.15, 0.7, 0.15])
    h2 = np.outer(k, k)
    blurred = db.convolve(h2, big)
    m1, m2 = big[10:80, 10:80], blurred[10:80, 10:80]
    zr = xr = (20, 51)
    f = db.window_filter(m1, m2, zr, xr, 11, 1e-6)
    res = (db.convolve(f, m2) - m1)[25:46, 25:46]
    base = (m2 - m1)[25:46, 25:46]
    assert np.linalg.norm(res) < 1e-3 * np.linalg.norm(base)
    # the filter's response at zero wavenumber undoes the blur's unit DC gain
    assert abs(f.sum() - 1.0) < 2e-3


def test_zero_plane_gives_zero():
    rng = np.random.default_rng(6)
    m = np.zeros((2, 30, 30))
    m[1] = rng.standard_normal((30, 30))
    out, F = db.deblur(m, m, spacing=10)
    assert np.all(out[0] == 0) and np.all(F[0] == 0)
    assert np.abs(out[1] - m[1]).max() < 1e-2 * np.abs(m[1]).max()


def test_nodes_and_windows_cover_the_image():
    for n, s in ((47, 10), (300, 20), (2000, 20), (11, 20)):
        zk = db.nodes(n, s)
        cover = np.zeros(n)
        for z in zk:
            cover += np.maximum(0.0, 1.0 - np.abs(np.arange(n) - z) / s)
        assert np.all(cover > 0)
