"""Pins of the oracle's muted data residuals (Sec. 4) and windowed modelling.

* the raised-cosine ramp: 0 / 0.5 / 1 at the start, middle and end of the
  taper, a hard step without taper;
* offsets from the geometry: |ix_r - ix_s| dx along a line, the hypotenuse in
  3D; the mask is symmetric in the offset sign and zero past the far-offset
  cut;
* in a homogeneous medium the direct-wave mute (v_mute = the medium's
  velocity, t0 = 2.5 / f0 covering the Ricker) removes the record down to
  the CPML and 2D-tail residue (< 0.5%);
* observed (two-layer) minus background (upper layer) data cancels the direct
  wave and keeps the reflection, which arrives after the mute at near
  offsets: the mask leaves it unchanged there;
* a window spanning the whole model is the plain modelling, bit for bit."""
import dataclasses

import numpy as np

import lsrtm_inputs as li
import oracle
from oracle import data as od


def test_ramp_closed_form():
    W = 0.04
    u = np.array([-1.0, 0.0, W / 2, W, 2 * W])
    assert np.allclose(od.ramp(u, W), [0.0, 0.0, 0.5, 1.0, 1.0], atol=1e-15)
    assert np.allclose(od.ramp(W / 4, W), 0.5 * (1 - np.cos(np.pi / 4)), atol=1e-15)
    assert np.array_equal(od.ramp(np.array([-1e-9, 0.0, 1e-9]), 0.0), [0.0, 0.0, 1.0])


def _line(nz=60, nx=161, nt=700, hetero=False):
    w = li.small_case(nz=nz, nx=nx, nt=nt, order=8, npml=20, nshot=1, seed=3, hetero=hetero, dx=10.0,
                      f0=20.0)
    w.geom = li.Geometry(np.array([1 * nx + 80], np.int32), np.array([0, nx], np.int32),
                         (1 * nx + np.arange(nx)).astype(np.int32))
    return w


def test_offsets_and_mask_geometry():
    w = _line(nt=400)
    o = od.offsets(w)
    assert np.allclose(o, np.abs(np.arange(w.nx) - 80) * w.dx)
    M = od.mute_mask(w, 2000.0, 0.01, 0.005, 400.0, 100.0)
    assert np.array_equal(M[80 - 30], M[80 + 30])       # symmetric in the offset sign
    assert np.all(M[o >= 400.0] == 0.0)
    assert np.all(M[o <= 300.0].max(axis=1) == 1.0)
    # each row is 0 up to the direct arrival, then rises monotonically
    t = (np.arange(w.nt) + 1) * w.dt
    for r in (70, 80, 95):
        td = o[r] / 2000.0 + 0.01
        assert np.all(M[r, t <= td] == 0.0)
        assert np.all(np.diff(M[r]) >= 0.0)
    # 3D: hypotenuse of the x and y offsets
    w3 = li.small_case(ndim=3, nz=6, ny=9, nx=11, nt=10, nshot=1, seed=2)
    w3.geom = li.Geometry(np.array([(1 * 9 + 4) * 11 + 5], np.int32), np.array([0, 2], np.int32),
                          np.array([(1 * 9 + 7) * 11 + 9, (2 * 9 + 4) * 11 + 5], np.int32))
    assert np.allclose(od.offsets(w3), [np.hypot(4 * w3.dx, 3 * w3.dy), 0.0])


def test_direct_wave_is_muted_in_a_homogeneous_medium():
    w = _line()
    d = oracle.model(w)
    f0 = 20.0
    M = od.mute_mask(w, 2000.0, 2.5 / f0, 0.25 / f0, 0.0, 0.0)
    assert np.linalg.norm(M * d) <= 5e-3 * np.linalg.norm(d)
    # without the wavelet allowance the direct wave is cut through and leaks
    M0 = od.mute_mask(w, 2000.0, 0.5 / f0, 0.25 / f0, 0.0, 0.0)
    assert np.linalg.norm(M0 * d) > 0.1 * np.linalg.norm(d)


def test_residual_keeps_the_near_offset_reflection():
    w = _line()
    vp2, rho2 = w.vp.copy(), w.rho.copy()
    vp2[30:], rho2[30:] = 2600.0, 2100.0
    vmax = 2600.0
    d_obs = oracle.model(w, vp=vp2, rho=rho2, vmax=vmax)
    d_bg = oracle.model(w, vmax=vmax)
    r = d_obs - d_bg
    f0, omax, otap = 20.0, 500.0, 100.0
    res = od.muted_residual(w, d_obs, d_bg, 2000.0, 2.0 / f0, 0.25 / f0, omax, otap)
    o = od.offsets(w)
    keep = o <= omax - otap
    assert np.linalg.norm((res - r)[keep]) <= 1e-6 * np.linalg.norm(r[keep])
    assert np.all(res[o >= omax] == 0.0)
    # the direct wave cancels in the residual: before the reflection (two-way
    # time 2 z / v at zero offset minus half the wavelet) it is ~0
    t = (np.arange(w.nt) + 1) * w.dt
    z = (30 - 1) * w.dx
    early = t < 2 * z / 2000.0 - 0.5 / f0
    assert np.abs(r[80, early]).max() <= 1e-6 * np.abs(d_obs[80]).max()


def test_full_width_window_models_like_the_plain_operator():
    w = li.small_case(nz=30, nx=50, nt=150, order=4, npml=8, nshot=2, seed=5)
    gw = dataclasses.replace(w.geom, win_x0=np.array([0, 0], np.int32), win_nx=np.array([50, 50], np.int32))
    assert np.array_equal(oracle.model(w, geom=gw), oracle.model(w))
