"""Interpolated PSF Hessian and image-domain CGNR (App. D) on the GPU against
the FP64 oracle.

* H x and H^T y on images spanning several tiles with ragged tails, 2D and 3D
  (Eq. trilinear with eight corners),
  every mask, default and extreme window half-widths: every output pixel;
* the dot test <H x, y> = <x, H^T y> on the GPU;
* PSFs from the oracle's own migration of a small survey (the real Hessian);
* CGNR: misfit history and solution after 10 iterations;
* the marine-line image size (300 x 2000, spacing 20, 1500 nodes per plane):
  sampled outputs computed one by one by the oracle (corners, edges, inside);
* host buffers through the C ABI, and argument errors."""
import ctypes

import numpy as np
import pytest

import lsrtm_inputs as li
import oracle
from oracle import psf_hessian as ph

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


def _f32(a):
    return np.asarray(a, np.float32).astype(np.float64)


def _dev(a):
    return None if a is None else torch.tensor(np.asarray(a, np.float32), device="cuda")


def _apply_gpu(h, x, pv, pi, s, half, mask, transpose):
    y = h.psf_hessian(_dev(x), _dev(pv), _dev(pi), s, half, transpose, mask)
    return y.double().cpu().numpy()


@pytest.mark.parametrize("nz,nx,s,half", [(70, 130, 10, -1), (90, 250, 20, -1), (41, 77, 6, 0), (75, 101, 32, 15)])
@pytest.mark.parametrize("mask", [1, 2, 3])
def test_apply_every_pixel(nz, nx, s, half, mask):
    pv, pi = li.psf_images(nz, nx, s, seed=nz + nx)
    pv, pi = _f32(pv), _f32(pi)
    x = _f32(np.random.default_rng(nz).standard_normal((2, nz, nx)))
    hh = ph.default_half(s) if half < 0 else half
    bl = ph.block_patches(pv if mask & 1 else None, pi if mask & 2 else None, s, hh, mask)
    h = _handle(nz, nx)
    for tr in (False, True):
        got = _apply_gpu(h, x, pv if mask & 1 else None, pi if mask & 2 else None, s, half, mask, tr)
        ref = ph.apply(bl, s, hh, x, transpose=tr)
        e = rel(got, ref)
        print(f"{nz}x{nx} s={s} half={hh} mask={mask} transpose={tr}: {e:.3e}")
        assert e < 1e-5
        for q in (0, 1):
            if not mask & (1 << q):
                assert np.all(got[q] == 0)
    h.close()


def test_dot_product_on_the_gpu():
    nz, nx, s = 96, 200, 16
    pv, pi = li.psf_images(nz, nx, s, seed=3)
    rng = np.random.default_rng(4)
    x = rng.standard_normal((2, nz, nx))
    y = rng.standard_normal((2, nz, nx))
    h = _handle(nz, nx)
    hx = _apply_gpu(h, x, pv, pi, s, -1, 3, False)
    hty = _apply_gpu(h, y, pv, pi, s, -1, 3, True)
    a = float(np.vdot(hx, _f32(y)))
    b = float(np.vdot(_f32(x), hty))
    print(f"<Hx,y> {a:.9e}  <x,H^T y> {b:.9e}")
    assert abs(a - b) <= 1e-5 * max(abs(a), abs(b))
    h.close()


def test_psfs_of_the_real_hessian():
    s = 10
    w = li.small_case(nz=40, nx=60, nt=260, order=4, npml=8, nshot=3, seed=41, nrec=40)
    pv = _f32(oracle.psf(w, 0, s))
    pi = _f32(oracle.psf(w, 1, s))
    x = _f32(oracle.adjoint(w, oracle.born(w, w.dm)))
    from paper_2508_10405_gb300 import Lsrtm
    h = Lsrtm.from_workload(w)
    bl = ph.block_patches(pv, pi, s, ph.default_half(s))
    for tr in (False, True):
        got = _apply_gpu(h, x, pv, pi, s, -1, 3, tr)
        ref = ph.apply(bl, s, ph.default_half(s), x, transpose=tr)
        print(f"real PSFs, transpose={tr}: {rel(got, ref):.3e}")
        assert rel(got, ref) < 1e-5
    h.close()


@pytest.mark.parametrize("mask", [2, 3])
def test_cgnr_against_the_oracle(mask):
    nz, nx, s, niter = 60, 110, 10, 10
    pv, pi = li.psf_images(nz, nx, s, seed=12)
    pv, pi = _f32(pv), _f32(pi)
    m_rtm, _ = li.image_pair(nz, nx, seed=13, nrefl=8)
    m_rtm = _f32(m_rtm)
    bl = ph.block_patches(pv if mask & 1 else None, pi, s, ph.default_half(s), mask)
    ref, mis_ref = ph.cgnr(bl, s, ph.default_half(s), m_rtm, niter, mask)
    h = _handle(nz, nx)
    got, mis = h.psf_cg(_dev(m_rtm), _dev(pv) if mask & 1 else None, _dev(pi), niter, s, -1, mask)
    got = got.double().cpu().numpy()
    print(f"mask {mask}: misfits {mis[-1]:.6f} / {mis_ref[-1]:.6f}, solution {rel(got, ref):.3e}")
    assert np.max(np.abs(mis - mis_ref)) < 1e-4
    assert mis[-1] < 0.5 * mis[0]
    assert rel(got, ref) < 1e-4
    h.close()


def test_marine_line_size_sampled():
    nz, nx, s = 300, 2000, 20
    half = ph.default_half(s)
    pv, pi = li.psf_images(nz, nx, s, seed=9)
    pv, pi = _f32(pv), _f32(pi)
    m_rtm, _ = li.image_pair(nz, nx, seed=5)
    x = _f32(m_rtm)
    bl = ph.block_patches(pv, pi, s, half)
    h = _handle(nz, nx)
    rng = np.random.default_rng(0)
    pix = [(0, 0), (0, nx - 1), (nz - 1, 0), (nz - 1, nx - 1), (9, 10), (10, 1990), (150, 1000), (299, 1234)]
    pix += [(int(z), int(x_)) for z, x_ in zip(rng.integers(0, nz, 16), rng.integers(0, nx, 16))]
    scale = None
    for tr in (False, True):
        got = _apply_gpu(h, x, pv, pi, s, -1, 3, tr)
        assert np.all(np.isfinite(got))
        scale = np.abs(got).max()
        for q in (0, 1):
            for z, xx in pix:
                ref = ph.apply_at(bl, s, half, x, q, z, xx, transpose=tr)
                assert abs(got[q, z, xx] - ref) <= 1e-5 * scale + 1e-5 * abs(ref), (tr, q, z, xx)
    h.close()


def test_host_buffers_through_the_c_abi():
    from paper_2508_10405_gb300 import binding
    nz, nx, s = 50, 70, 10
    pv, pi = li.psf_images(nz, nx, s, seed=21)
    pv32, pi32 = np.ascontiguousarray(pv, np.float32), np.ascontiguousarray(pi, np.float32)
    x = np.ascontiguousarray(np.random.default_rng(2).standard_normal((2, nz, nx)), np.float32)
    h = _handle(nz, nx)
    y = np.zeros_like(x)
    rc = h._lib.lsrtm_psf_hessian(h._h, binding._ptr(pv32), binding._ptr(pi32), s, -1, 3, 0,
                                  binding._ptr(x), binding._ptr(y))
    assert rc == 0
    bl = ph.block_patches(_f32(pv32), _f32(pi32), s, ph.default_half(s))
    assert rel(y, ph.apply(bl, s, ph.default_half(s), _f32(x))) < 1e-5
    dm = np.zeros_like(x)
    mis = (ctypes.c_double * 6)()
    rc = h._lib.lsrtm_psf_cg(h._h, binding._ptr(pv32), binding._ptr(pi32), s, -1, 3, binding._ptr(x),
                             binding._ptr(dm), 5, mis)
    assert rc == 0
    ref, mis_ref = ph.cgnr(bl, s, ph.default_half(s), _f32(x), 5)
    assert rel(dm, ref) < 1e-4 and abs(mis[5] - mis_ref[5]) < 1e-4
    h.close()


def test_argument_errors():
    from paper_2508_10405_gb300 import LsrtmError
    nz, nx = 30, 40
    h = _handle(nz, nx)
    a = torch.zeros((2, nz, nx), device="cuda")
    b = torch.zeros((2, nz, nx), device="cuda")
    for kw in (dict(spacing=1), dict(spacing=65), dict(half=16), dict(param_mask=0), dict(param_mask=4)):
        args = dict(spacing=10, half=-1, param_mask=3)
        args.update(kw)
        with pytest.raises(LsrtmError):
            h.psf_hessian(a, b, b, args["spacing"], args["half"], False, args["param_mask"])
    with pytest.raises(LsrtmError):
        h.psf_hessian(a, None, b, 10, -1, False, 3)            # Vp in the mask, no Vp PSF
    with pytest.raises(LsrtmError):
        h.psf_hessian(a, b, b, 10, -1, False, 3, out=a)        # x and y overlap
    with pytest.raises(LsrtmError):
        h.psf_hessian(a, b, b, 62, -1, False, 3)               # no comb node in a 30-row image
    with pytest.raises(LsrtmError):
        h.psf_cg(a, b, b, -1, 10)
    h.close()


# ------------------------------------------------------------------ 3D

def _handle3(shape):
    from paper_2508_10405_gb300 import Lsrtm
    nz, ny, nx = shape
    w = li.small_case(ndim=3, nz=nz, ny=ny, nx=nx, nt=8, order=4, npml=4, nshot=1, seed=1)
    return Lsrtm.from_workload(w)


@pytest.mark.parametrize("shape,s,half", [((20, 14, 26), 6, -1), ((17, 21, 45), 8, 2)])
@pytest.mark.parametrize("mask", [1, 2, 3])
def test_apply_3d_every_voxel(shape, s, half, mask):
    pv, pi = li.psf_images3(*shape, s, seed=sum(shape))
    pv, pi = _f32(pv), _f32(pi)
    x = _f32(np.random.default_rng(3).standard_normal((2,) + shape))
    hh = ph.default_half(s) if half < 0 else half
    bl = ph.block_patches(pv if mask & 1 else None, pi if mask & 2 else None, s, hh, mask)
    h = _handle3(shape)
    for tr in (False, True):
        got = _apply_gpu(h, x, pv if mask & 1 else None, pi if mask & 2 else None, s, half, mask, tr)
        ref = ph.apply(bl, s, hh, x, transpose=tr)
        e = rel(got, ref)
        print(f"3D {shape} s={s} half={hh} mask={mask} transpose={tr}: {e:.3e}")
        assert e < 1e-5
        for q in (0, 1):
            if not mask & (1 << q):
                assert np.all(got[q] == 0)
    h.close()


def test_cgnr_and_dot_product_3d():
    shape, s, niter = (18, 15, 22), 6, 6
    pv, pi = li.psf_images3(*shape, s, seed=5)
    pv, pi = _f32(pv), _f32(pi)
    rng = np.random.default_rng(6)
    m_rtm = _f32(rng.standard_normal((2,) + shape))
    h = _handle3(shape)
    x = rng.standard_normal((2,) + shape)
    y = rng.standard_normal((2,) + shape)
    a = float(np.vdot(_apply_gpu(h, x, pv, pi, s, -1, 3, False), _f32(y)))
    b = float(np.vdot(_f32(x), _apply_gpu(h, y, pv, pi, s, -1, 3, True)))
    assert abs(a - b) <= 1e-5 * max(abs(a), abs(b))
    bl = ph.block_patches(pv, pi, s, ph.default_half(s))
    ref, mis_ref = ph.cgnr(bl, s, ph.default_half(s), m_rtm, niter)
    got, mis = h.psf_cg(_dev(m_rtm), _dev(pv), _dev(pi), niter, s)
    print(f"3D CGNR: misfit {mis[-1]:.6f} / {mis_ref[-1]:.6f}, solution {rel(got.double().cpu().numpy(), ref):.3e}")
    assert np.max(np.abs(mis - mis_ref)) < 1e-4
    assert rel(got.double().cpu().numpy(), ref) < 1e-4
    h.close()
