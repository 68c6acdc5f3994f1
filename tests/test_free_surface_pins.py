"""Pins of the oracle's free surface (method of images on the first interior
row) against facts that do not come from the free-surface code:

  * the method of images itself: in a homogeneous medium the free-surface
    field equals the full-space field of the source minus that of its mirror
    source, computed by the (separately pinned) full-space operator on a
    domain symmetric about the surface row;
  * the closed-form 2D half-space Green's function G(r1) - G(r2);
  * p = 0 on the surface: receivers there record exactly zero;
  * L^T stays the exact transpose (dot test, explicit matrices on a tiny
    grid) and L the Jacobian of nonlinear modelling (linearisation slope)."""
import dataclasses

import numpy as np
import pytest

import lsrtm_inputs as li
import oracle
from lsrtm_inputs import Geometry, Workload
from tests import analytic


def _homog(nz, nx, npml, dx, dt, nt, order, f0, delay, srcs, recs, fs, v=2000.0, rho=1000.0):
    shape = (nz, nx)
    geom = Geometry(np.array([srcs[0]], np.int32), np.array([0, len(recs)], np.int32),
                    np.asarray(recs, np.int32))
    return Workload("homog_fs", 2, nz, 1, nx, dx, dx, dx, dt, nt, order, npml, f0,
                    np.full(shape, v), np.full(shape, rho), np.zeros((2,) + shape),
                    li.ricker(nt, dt, f0, delay), geom, free_surface=fs)


@pytest.mark.parametrize("order", [4, 8])
def test_free_surface_equals_mirror_source_superposition(order):
    """Free-surface records in a homogeneous medium = full-space records of the
    source minus those of its mirror about the surface row, the full-space
    grid being the free-surface grid reflected about that row (so its CPML is
    symmetric too): the discrete method of images, exact to rounding."""
    nz, nx, npml, dx, dt, nt = 40, 60, 12, 10.0, 1e-3, 260
    zs_src, xs = 6, 30
    rec = [(0, 20), (1, 20), (3, 45), (9, 12), (25, 30)]
    w = _homog(nz, nx, npml, dx, dt, nt, order, 15.0, 0.1, [zs_src * nx + xs],
               [z * nx + x for z, x in rec], fs=True)
    d_fs = oracle.model(w, vmax=2000.0)
    # full space: interior rows -(nz-1) .. nz-1 around the surface row nz-1
    nzf = 2 * nz - 1
    s = nz - 1
    wf = _homog(nzf, nx, npml, dx, dt, nt, order, 15.0, 0.1, [(s + zs_src) * nx + xs],
                [(s + z) * nx + x for z, x in rec], fs=False)
    d1 = oracle.model(wf, vmax=2000.0)
    wm = dataclasses.replace(wf, geom=Geometry(np.array([(s - zs_src) * nx + xs], np.int32),
                                                wf.geom.rec_ptr, wf.geom.rec_idx))
    d2 = oracle.model(wm, vmax=2000.0)
    ref = d1 - d2
    assert np.abs(ref).max() > 0
    np.testing.assert_allclose(d_fs, ref, rtol=0, atol=1e-11 * np.abs(ref).max())
    # the surface row records nothing
    assert np.all(d_fs[0] == 0.0)


def _half_space_error(dx, dt, nt):
    n = int(round(121 * 10 / dx))
    f0, delay, c = 12.0, 1.5 / 12.0, 2000.0
    zsrc, xsrc = int(round(100 / dx)), n // 2
    zrec, xrec = zsrc, n // 2 + int(round(400 / dx))
    w = _homog(n, n, 20, dx, dt, nt, 8, f0, delay, [zsrc * n + xsrc], [zrec * n + xrec], fs=True, v=c)
    d = oracle.model(w, vmax=c)[0]
    t = (np.arange(nt) + 1) * dt
    r1 = np.hypot((zrec - zsrc) * dx, (xrec - xsrc) * dx)
    r2 = np.hypot((zrec + zsrc) * dx, (xrec - xsrc) * dx)
    # injection of w(n dt) over step n acts as the source s(t) = w(t - dt/2)
    ref = analytic.green2d_pressure(r1, t, c, f0, delay + dt / 2) - \
        analytic.green2d_pressure(r2, t, c, f0, delay + dt / 2)
    w0 = dataclasses.replace(w, free_surface=False)
    d0 = oracle.model(w0, vmax=c)[0]
    return (np.linalg.norm(d - ref) / np.linalg.norm(ref),
            np.linalg.norm(d0 - ref) / np.linalg.norm(ref))


def test_free_surface_half_space_green_function():
    """2D half-space response G(r1) - G(r2) (line-source Green's function and
    its negative image, source 100 m below the surface, receiver 400 m away at
    the same depth): second-order convergence, as the full-space pin; without
    the free surface the receiver sees only the direct wave."""
    e10, e10_nofs = _half_space_error(10.0, 1e-3, 300)
    e5, _ = _half_space_error(5.0, 0.5e-3, 600)
    assert e10 < 1.5e-2 and e5 < 4e-3, (e10, e5)
    assert e10 / e5 > 3.5, (e10, e5)
    assert e10_nofs > 0.3, e10_nofs


def _fs_case(ndim, order, **kw):
    base = (dict(nz=20, nx=24, nt=120, npml=8, nshot=3) if ndim == 2 else
            dict(ndim=3, nz=10, ny=9, nx=12, nt=50, npml=5, nshot=2))
    base.update(kw)
    w = li.small_case(order=order, seed=order + 40, **base)
    return dataclasses.replace(w, free_surface=True)


@pytest.mark.parametrize("ndim,order", [(2, 4), (2, 8), (3, 4), (3, 8)])
def test_free_surface_dot_product(ndim, order):
    """<L m, d> = <m, L^T d> to 1e-12 with the free surface, including
    receivers on the surface row."""
    w = _fs_case(ndim, order)
    nx = w.nx
    idx = w.geom.rec_idx.copy()
    idx[0] = idx[0] % (w.nx * w.ny)   # first receiver moved onto the surface row
    w = dataclasses.replace(w, geom=Geometry(w.geom.src_idx, w.geom.rec_ptr, idx))
    rng = np.random.default_rng(200 + ndim * 10 + order)
    m = rng.standard_normal((2,) + w.shape)
    d = rng.standard_normal((w.geom.nrec_total, w.nt))
    Lm = oracle.born(w, m)
    assert np.all(Lm[0] == 0.0)   # the surface receiver records nothing
    a = float(np.vdot(Lm, d))
    b = float(np.vdot(m, oracle.adjoint(w, d)))
    assert abs(a - b) / max(abs(a), abs(b)) < 1e-12, (a, b)


def test_free_surface_explicit_matrices_tiny():
    """The matrix of L^T equals the transpose of the matrix of L, both built
    column by column, with the free surface."""
    w = dataclasses.replace(li.small_case(nz=5, nx=6, nt=18, order=4, npml=3, nshot=1, seed=3, nrec=3),
                            free_surface=True)
    n2, nd = 2 * w.nint, w.geom.nrec_total * w.nt
    L = np.zeros((nd, n2))
    for j in range(n2):
        e = np.zeros(n2)
        e[j] = 1.0
        L[:, j] = oracle.born(w, e.reshape((2,) + w.shape)).ravel()
    LT = np.zeros((n2, nd))
    for i in range(nd):
        e = np.zeros(nd)
        e[i] = 1.0
        LT[:, i] = oracle.adjoint(w, e.reshape(w.geom.nrec_total, w.nt)).ravel()
    scale = np.abs(L).max()
    assert scale > 0
    np.testing.assert_allclose(LT, L.T, rtol=0, atol=1e-12 * scale)


@pytest.mark.parametrize("ndim", [2, 3])
def test_free_surface_linearisation(ndim):
    """F(m0 + eps dm) - F(m0) - eps L dm = O(eps^2) with the free surface."""
    w = (_fs_case(2, 4, nz=22, nx=26, nt=140, npml=6, nshot=2) if ndim == 2
         else _fs_case(3, 4, nz=10, ny=9, nx=11, nt=60, npml=4, nshot=1))
    dm = w.dm
    vmax = float(np.max(w.vp))
    F0 = oracle.model(w, vmax=vmax)
    Ldm = oracle.born(w, dm, vmax=vmax)
    errs = []
    for eps in (1e-2, 1e-3):
        F1 = oracle.model(w, vp=w.vp * np.exp(eps * dm[0]), rho=w.rho * np.exp(eps * (dm[1] - dm[0])),
                          vmax=vmax)
        errs.append(np.linalg.norm(F1 - F0 - eps * Ldm) / np.linalg.norm(eps * Ldm))
    assert errs[1] < 5e-3, errs
    assert 8.0 < errs[0] / errs[1] < 12.5, errs
