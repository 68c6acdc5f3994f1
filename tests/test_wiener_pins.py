"""Pins of the oracle's nonstationary Wiener filter (App. E, Fourier form).

* numpy's fft2 is the DFT written out as a sum (sign and index convention);
* the Wiener ratio minimises the paper's per-wavenumber objective
  |[F m']_i - l [F m'']_i|^2 + eps |l|^2: every perturbed l does worse (a
  conjugate on the wrong factor fails);
* a block blurred by a circular convolution (written as a brute-force sum)
  is deconvolved exactly as eps -> 0: re-blurring the result gives the block;
* m'' = c m' gives dm = m_rtm / c everywhere (blocks and valence blend), the
  identity for c = 1;
* a zero m'' plane (mono-parameter) gives a zero plane."""
import numpy as np
import pytest

from oracle import wiener as wf


def _dft2(x):
    n, m = x.shape
    k = np.arange(n)[:, None]
    l = np.arange(m)[None, :]
    out = np.zeros((n, m), complex)
    for a in range(n):
        for b in range(m):
            out += x[a, b] * np.exp(-2j * np.pi * (k * a / n + l * b / m))
    return out


def test_fft2_is_the_dft_sum():
    x = np.random.default_rng(0).standard_normal((6, 4))
    assert np.allclose(np.fft.fft2(x), _dft2(x), atol=1e-12)


def test_wiener_ratio_minimises_the_objective():
    rng = np.random.default_rng(1)
    m1 = rng.standard_normal((8, 8))
    m2 = rng.standard_normal((8, 8))
    eps = 0.3
    lam = wf.inverse_eigenvalues(m1, m2, eps)
    A, B = _dft2(m2), _dft2(m1)
    eps_k = eps * np.mean(np.abs(A) ** 2)
    J = lambda l: np.abs(B - l * A) ** 2 + eps_k * np.abs(l) ** 2
    j0 = J(lam)
    for d in (1e-3, -1e-3, 1e-3j, -1e-3j, 1e-3 + 1e-3j):
        assert np.all(J(lam + d) > j0)
    # the closed form against the normal equation of each wavenumber
    assert np.allclose((np.abs(A) ** 2 + eps_k) * lam, np.conj(A) * B, atol=1e-10)


def test_circular_blur_is_deconvolved_in_a_block():
    s = 6
    n = 2 * s
    rng = np.random.default_rng(2)
    b = rng.standard_normal((n, n))
    h = np.zeros((n, n))
    h[0, 0], h[1, 0], h[-1, 0], h[0, 1], h[0, -1] = 0.6, 0.1, 0.1, 0.1, 0.1
    blur = lambda g: np.array([[sum(g[(i - a) % n, (j - c) % n] * h[a, c] for a in range(n) for c in range(n))
                                for j in range(n)] for i in range(n)])
    out = wf.block_filter(b, blur(b), 1e-14)
    assert np.allclose(blur(out), b, atol=1e-8)


@pytest.mark.parametrize("c", [1.0, 2.5])
def test_scaled_remigration_gives_the_scaled_image(c):
    rng = np.random.default_rng(3)
    m = rng.standard_normal((2, 37, 53))
    out = wf.wiener(m, c * m, 10, eps=1e-13)
    assert np.allclose(out, m / c, atol=1e-7)


def test_zero_remigrated_plane_gives_zero():
    rng = np.random.default_rng(4)
    m = rng.standard_normal((2, 30, 40))
    r = rng.standard_normal((2, 30, 40))
    r[0] = 0.0
    out = wf.wiener(m, r, 8, eps=1e-3)
    assert np.all(out[0] == 0.0) and np.any(out[1] != 0.0)
