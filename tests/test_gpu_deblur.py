"""Deblurring filters (App. E) on the GPU against the FP64 oracle.

* small images: every filter and every output pixel;
* images from the oracle's own migration and remigration of a small survey
  (the real Hessian blur), both parameters and the mono-parameter (Ip) case;
* the marine-line image size (300 x 2000, spacing 20, 11 x 11 filters, 1500
  nodes per plane) through the C ABI: the oracle runs on crops whose origin is
  on the node grid, so the crops' nodes away from the cut edges have the same
  windows as the full image, and their filters and the pixels they cover
  must match the GPU's full-size result (one crop on the image's top-right
  corner, one inside)."""
import numpy as np
import pytest

import lsrtm_inputs as li
import oracle
from oracle import deblur as db

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


def _gpu(h, a, b, s, flen, eps):
    out, F = h.deblur(torch.tensor(a, dtype=torch.float32, device="cuda"),
                      torch.tensor(b, dtype=torch.float32, device="cuda"), s, flen, eps,
                      return_filters=True)
    return out.double().cpu().numpy(), F.double().cpu().numpy()


@pytest.mark.parametrize("nz,nx,s,flen,eps", [(47, 61, 10, 11, 1e-3), (33, 29, 8, 5, 1e-2),
                                               (40, 52, 6, 7, 0.0)])
def test_small_images_every_filter_and_pixel(nz, nx, s, flen, eps):
    m, r = li.image_pair(nz, nx, seed=nz + nx, nrefl=6)
    m = m.astype(np.float32).astype(np.float64)
    r = r.astype(np.float32).astype(np.float64)
    h = _handle(nz, nx)
    out, F = _gpu(h, m, r, s, flen, eps)
    ref, Fr = db.deblur(m, r, s, flen, eps)
    print(f"{nz}x{nx} s={s} flen={flen}: filters {rel(F, Fr):.3e}, image {rel(out, ref):.3e}")
    assert rel(F, Fr) < 1e-5
    assert rel(out, ref) < 1e-5
    h.close()


def test_hessian_images_two_parameter_and_mono():
    w = li.small_case(nz=40, nx=60, nt=260, order=4, npml=8, nshot=3, seed=41, nrec=40)
    d = oracle.born(w, w.dm)
    m_rtm = oracle.adjoint(w, d)
    m_rem = oracle.remigrate(w, m_rtm)
    m_rtm = m_rtm.astype(np.float32).astype(np.float64)
    m_rem = m_rem.astype(np.float32).astype(np.float64)
    from paper_2508_10405_gb300 import Lsrtm
    h = Lsrtm.from_workload(w)
    out, F = _gpu(h, m_rtm, m_rem, 10, 11, 1e-3)
    ref, Fr = db.deblur(m_rtm, m_rem, 10, 11, 1e-3)
    print(f"Hessian images: filters {rel(F, Fr):.3e}, image {rel(out, ref):.3e}")
    assert rel(F, Fr) < 1e-5 and rel(out, ref) < 1e-5
    # mono-parameter (Ip): the zero Vp plane gets zero filters and a zero image
    m1 = m_rtm.copy()
    m1[0] = 0
    r1 = m_rem.copy()
    r1[0] = 0
    out1, F1 = _gpu(h, m1, r1, 10, 11, 1e-3)
    assert np.all(out1[0] == 0) and np.all(F1[0] == 0)
    assert rel(out1[1], ref[1]) < 1e-5
    h.close()


def _crop_check(out, F, m, r, z0, z1, x0, x1, s, flen, eps):
    """Oracle on m[:, z0:z1, x0:x1] (origin on the node grid); compare the
    filters of nodes whose window + taps stay inside the crop, and the pixels
    covered only by such nodes (where the crop's cut edges are real image
    edges, everything up to them counts)."""
    nz, nx = m.shape[1:]
    h = flen // 2
    ref, Fr = db.deblur(m[:, z0:z1, x0:x1], r[:, z0:z1, x0:x1], s, flen, eps)
    zk = db.nodes(z1 - z0, s) + z0
    xk = db.nodes(x1 - x0, s) + x0
    okz = [(z0 == 0 or z - s - h >= z0) and (z1 == nz or z + s + h < z1) for z in zk]
    okx = [(x0 == 0 or x - s - h >= x0) and (x1 == nx or x + s + h < x1) for x in xk]
    iz = np.flatnonzero(okz)
    ix = np.flatnonzero(okx)
    gz = (zk[iz] - s // 2) // s
    gx = (xk[ix] - s // 2) // s
    Fg = F[:, gz][:, :, gx]
    Fo = Fr[:, iz][:, :, ix]
    zlo = 0 if z0 == 0 else zk[iz[0]]
    zhi = nz if z1 == nz else zk[iz[-1]] + 1
    xlo = 0 if x0 == 0 else xk[ix[0]]
    xhi = nx if x1 == nx else xk[ix[-1]] + 1
    og = out[:, zlo:zhi, xlo:xhi]
    oo = ref[:, zlo - z0:zhi - z0, xlo - x0:xhi - x0]
    return rel(Fg, Fo), rel(og, oo), len(iz) * len(ix)


def test_marine_line_size_on_crops():
    nz, nx, s, flen, eps = 300, 2000, 20, 11, 1e-3
    m, r = li.image_pair(nz, nx, seed=5)
    m = m.astype(np.float32).astype(np.float64)
    r = r.astype(np.float32).astype(np.float64)
    h = _handle(nz, nx)
    out, F = _gpu(h, m, r, s, flen, eps)
    assert F.shape == (2, 15, 100, flen, flen)
    assert np.all(np.isfinite(out))
    for crop in ((0, 120, 1880, 2000), (140, 300, 900, 1060)):
        ef, eo, nn = _crop_check(out, F, m, r, *crop, s, flen, eps)
        print(f"crop {crop}: {nn} nodes, filters {ef:.3e}, image {eo:.3e}")
        assert nn >= 9
        assert ef < 1e-5 and eo < 1e-5
    h.close()


def test_argument_errors():
    from paper_2508_10405_gb300 import LsrtmError
    h = _handle(30, 30)
    a = torch.zeros((2, 30, 30), device="cuda")
    for kw in (dict(flen=4), dict(flen=13), dict(spacing=1), dict(spacing=49), dict(eps=-1.0)):
        args = dict(spacing=10, flen=11, eps=1e-3)
        args.update(kw)
        with pytest.raises(LsrtmError):
            h.deblur(a, a, **args)
    h.close()


def test_windowed_handle_filters_the_model_sized_image():
    """Handles with per-shot aperture windows run their wavefields on the
    widest window's grid; the deblurring works on the model-sized image."""
    import dataclasses
    from paper_2508_10405_gb300 import Lsrtm
    w = li.preset(5, nz=36, nx=110, nt=8, nshot=4, shot_dx=22, shot_x0=8, nrec_range=(6, 14), margin=9)
    w = dataclasses.replace(w, npml=10)
    assert np.all(w.geom.win_nx < w.nx)
    m, r = li.image_pair(36, 110, seed=7, nrefl=6)
    m = m.astype(np.float32).astype(np.float64)
    r = r.astype(np.float32).astype(np.float64)
    h = Lsrtm.from_workload(w)
    out, F = _gpu(h, m, r, 10, 7, 1e-3)
    ref, Fr = db.deblur(m, r, 10, 7, 1e-3)
    assert out.shape == (2, 36, 110)
    assert rel(F, Fr) < 1e-5 and rel(out, ref) < 1e-5
    h.close()
