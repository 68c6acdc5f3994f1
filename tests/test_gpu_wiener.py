"""Nonstationary Wiener deblurring (App. E, Fourier form) on the GPU against
the FP64 oracle, every output pixel:

* small images with ragged node grids, several spacings and stabilisers;
* images from the oracle's own migration and remigration of a small survey
  (the real Hessian blur), both parameters and the mono-parameter (Ip) case;
* the marine-line image size (300 x 2000, spacing 20: 1500 blocks of 40 x 40
  per plane) through device buffers, and host buffers through the C ABI;
* m'' = c m' returns m_rtm / c; argument errors."""
import numpy as np
import pytest

import lsrtm_inputs as li
import oracle
from oracle import wiener as wf

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _handle(nz, nx):
    from paper_2508_10405_gb300 import Lsrtm
    w = li.small_case(nz=nz, nx=nx, nt=8, order=4, npml=4, nshot=1, seed=1)
    return Lsrtm.from_workload(w)


def _gpu(h, a, b, s, eps):
    out = h.deblur_wiener(torch.tensor(a, dtype=torch.float32, device="cuda"),
                          torch.tensor(b, dtype=torch.float32, device="cuda"), s, eps)
    return out.double().cpu().numpy()


def _f32(a):
    return np.asarray(a, np.float32).astype(np.float64)


@pytest.mark.parametrize("nz,nx,s,eps", [(47, 61, 10, 1e-3), (33, 29, 8, 1e-2), (40, 52, 6, 1e-3), (70, 130, 32, 1e-3),
                                         (9, 14, 2, 1e-2)])
def test_small_images_every_pixel(nz, nx, s, eps):
    m, r = li.image_pair(nz, nx, seed=nz + nx, nrefl=6)
    m, r = _f32(m), _f32(r)
    h = _handle(nz, nx)
    got = _gpu(h, m, r, s, eps)
    ref = wf.wiener(m, r, s, eps)
    print(f"{nz}x{nx} s={s} eps={eps}: {rel(got, ref):.3e}")
    assert rel(got, ref) < 2e-4
    h.close()


def test_hessian_images_two_parameter_and_mono():
    w = li.small_case(nz=40, nx=60, nt=260, order=4, npml=8, nshot=3, seed=41, nrec=40)
    m_rtm = oracle.adjoint(w, oracle.born(w, w.dm))
    m_rem = _f32(oracle.remigrate(w, m_rtm))
    m_rtm = _f32(m_rtm)
    from paper_2508_10405_gb300 import Lsrtm
    h = Lsrtm.from_workload(w)
    got = _gpu(h, m_rtm, m_rem, 10, 1e-3)
    ref = wf.wiener(m_rtm, m_rem, 10, 1e-3)
    print(f"Hessian images: {rel(got, ref):.3e}")
    assert rel(got, ref) < 2e-4
    m1, r1 = m_rtm.copy(), m_rem.copy()
    m1[0] = 0.0
    r1[0] = 0.0
    got1 = _gpu(h, m1, r1, 10, 1e-3)
    assert np.all(got1[0] == 0.0)
    assert rel(got1[1], ref[1]) < 2e-4
    h.close()


def test_marine_line_size():
    nz, nx, s = 300, 2000, 20
    m, r = li.image_pair(nz, nx, seed=5)
    m, r = _f32(m), _f32(r)
    h = _handle(nz, nx)
    got = _gpu(h, m, r, s, 1e-3)
    ref = wf.wiener(m, r, s, 1e-3)
    print(f"marine line: {rel(got, ref):.3e}")
    assert np.all(np.isfinite(got)) and rel(got, ref) < 2e-4
    # host buffers through the C ABI
    from paper_2508_10405_gb300 import binding
    a = np.ascontiguousarray(m, np.float32)
    b = np.ascontiguousarray(r, np.float32)
    out = np.zeros_like(a)
    assert h._lib.lsrtm_deblur_wiener(h._h, binding._ptr(a), binding._ptr(b), s, 1e-3, binding._ptr(out)) == 0
    assert np.array_equal(out.astype(np.float64), got)
    h.close()


def test_scaled_remigration():
    m = np.random.default_rng(3).standard_normal((2, 37, 53)).astype(np.float32).astype(np.float64)
    h = _handle(37, 53)
    got = _gpu(h, m, 2.0 * m, 10, 1e-9)
    assert np.max(np.abs(got - m / 2.0)) < 1e-3 * np.max(np.abs(m))
    h.close()


def test_argument_errors():
    from paper_2508_10405_gb300 import LsrtmError
    h = _handle(30, 30)
    a = torch.zeros((2, 30, 30), device="cuda")
    for s, eps in ((1, 1e-3), (33, 1e-3), (10, 0.0), (10, -1.0), (10, float("nan")), (62, 1e-3)):
        with pytest.raises(LsrtmError):
            h.deblur_wiener(a, a, s, eps)
    h.close()
