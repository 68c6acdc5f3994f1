"""Pins of the FP64 oracle against facts that do not come from the oracle:
textbook coefficients, closed-form wave solutions, reflection coefficients,
the Jacobian of nonlinear modelling, exact transposition, dense least squares.

Each test targets a plausible mistake: a dropped Born term or wrong sign
(linearisation), a wrong buoyancy or density use (reflection coefficient of a
density-only contrast), a wrong time/space index or scaling (Green's
functions, point scatterer), a wrong transposed sub-step (dot test, explicit
matrices), a broken solver (least squares)."""
import math

import numpy as np
import pytest

import lsrtm_inputs as li
import oracle
from lsrtm_inputs import Geometry, Workload
from tests import analytic


def _homog_workload(ndim, n, npml, dx, dt, nt, order, f0, delay, src, recs, v=2000.0,
                    rho=1000.0):
    shape = (n, n) if ndim == 2 else (n, n, n)
    ny = n if ndim == 3 else 1
    geom = Geometry(np.array([src], np.int32), np.array([0, len(recs)], np.int32),
                    np.asarray(recs, np.int32))
    return Workload("homog", ndim, n, ny, n, dx, dx, dx, dt, nt, order, npml, f0,
                    np.full(shape, v), np.full(shape, rho), np.zeros((2,) + shape),
                    li.ricker(nt, dt, f0, delay), geom)


# ---------------------------------------------------------------- FD coeffs

def test_fd_coefficients_textbook():
    # Staggered-grid Taylor coefficients (Levander 1988 for order 4; order 8
    # from the same Taylor conditions): closed forms.
    np.testing.assert_allclose(oracle.fd_coeffs(4), [9 / 8, -1 / 24], rtol=0, atol=1e-15)
    np.testing.assert_allclose(oracle.fd_coeffs(8),
                               [1225 / 1024, -245 / 3072, 49 / 5120, -5 / 7168],
                               rtol=0, atol=1e-14)


# ---------------------------------------------------------- Green's functions

@pytest.mark.parametrize("dx,dt,nt,tol", [(10.0, 1e-3, 300, 1.2e-2), (5.0, 0.5e-3, 600, 3e-3)])
def test_green_2d_homogeneous(dx, dt, nt, tol):
    """Eq. (1) with a point pressure source in 2D reproduces the line-source
    Green's function convolved with s'; error falls at second order."""
    n = int(round(121 * 10 / dx))
    f0, delay, c = 12.0, 1.5 / 12.0, 2000.0
    mid = n // 2
    off = int(round(400 / dx))
    w = _homog_workload(2, n, 20, dx, dt, nt, 8, f0, delay, mid * n + mid, [mid * n + mid + off])
    d = oracle.model(w)[0]
    t = (np.arange(nt) + 1) * dt
    # injection of w(n dt) over step n acts as the source s(t) = w(t - dt/2)
    ref = analytic.green2d_pressure(off * dx, t, c, f0, delay + dt / 2)
    err = np.linalg.norm(d - ref) / np.linalg.norm(ref)
    assert err < tol, err


def test_green_3d_homogeneous():
    dx, dt, nt, n, f0, c = 10.0, 1e-3, 200, 41, 12.0, 2000.0
    delay = 1.5 / f0
    mid = n // 2
    off = 14
    src = (mid * n + mid) * n + mid
    w = _homog_workload(3, n, 10, dx, dt, nt, 8, f0, delay, src, [src + off])
    d = oracle.model(w)[0]
    t = (np.arange(nt) + 1) * dt
    ref = analytic.green3d_pressure(off * dx, t, c, f0, delay + dt / 2)
    err = np.linalg.norm(d - ref) / np.linalg.norm(ref)
    assert err < 1.2e-2, err


def test_cpml_absorbs():
    """A trace in a small CPML box matches the same trace in a box large enough
    that no boundary signal arrives in the window (boundary reflections of
    the absorbing strips stay below 1%)."""
    dx, dt, nt, f0, order = 10.0, 1e-3, 450, 12.0, 8
    delay = 1.5 / f0
    traces = []
    for n in (61, 181):
        mid = n // 2
        src = mid * n + mid
        w = _homog_workload(2, n, 20, dx, dt, nt, order, f0, delay, src, [src + 10])
        traces.append(oracle.model(w)[0])
    err = np.linalg.norm(traces[0] - traces[1]) / np.linalg.norm(traces[1])
    assert err < 1e-2, err


# ---------------------------------------------------- reflection coefficient

def _plane_wave_R(v1, r1, v2, r2):
    dx, dt, nt, f0 = 5.0, 0.4e-3, 1100, 15.0
    nz, nx, zi, zs, zr = 130, 400, 100, 40, 60
    vp = np.full((nz, nx), float(v1))
    rho = np.full((nz, nx), float(r1))
    vp[zi:] = v2
    rho[zi:] = r2
    delay = 1.5 / f0
    cx = nx // 2
    geom = Geometry(np.array([zs * nx + cx], np.int32), np.array([0, 1], np.int32),
                    np.array([zr * nx + cx], np.int32))
    w = Workload("refl", 2, nz, 1, nx, dx, dx, dx, dt, nt, 8, 20, f0, vp, rho,
                 np.zeros((2, nz, nx)), li.ricker(nt, dt, f0, delay), geom)
    line = np.array([zs * nx + x for x in range(nx)], np.int32)
    d = oracle.model(w, src_ptr=np.array([0, nx], np.int32), src_idx=line)[0]
    t = (np.arange(nt) + 1) * dt
    td = (zr - zs) * dx / v1 + delay
    tr = (2 * (zi - 0.5) - zs - zr) * dx / v1 + delay
    half = 1.2 / f0
    md, mr = np.abs(t - td) < half, np.abs(t - tr) < half
    a_d = d[md][np.argmax(np.abs(d[md]))]
    a_r = d[mr][np.argmax(np.abs(d[mr]))]
    return a_r / a_d


@pytest.mark.parametrize("case", [(2000, 1000, 3000, 1000), (2000, 1000, 2000, 1500),
                                  (2000, 1500, 1600, 1000)])
def test_normal_incidence_reflection(case):
    """A plane wave from a line source reflects off a flat interface with
    R = (Z2 - Z1)/(Z2 + Z1), Z = rho v: pins how density and velocity enter
    Eq. (1) (a velocity-only and a density-only contrast give the same R)."""
    v1, r1, v2, r2 = case
    R = _plane_wave_R(v1, r1, v2, r2)
    exact = (v2 * r2 - v1 * r1) / (v2 * r2 + v1 * r1)
    assert abs(R - exact) < 4e-3, (R, exact)


# --------------------------------------------------------- Born scattering

def test_born_3d_point_scatterer():
    """Born response of a single dln kappa spike (dln Vp = dln Ip = a/2, so
    dln rho = 0) in a homogeneous medium equals a V s'''(t-(r1+r2)/c) /
    (16 pi^2 c^4 r1 r2): pins the kappa term of Eq. (scattereqln)."""
    dx, dt, nt, n, f0, v = 10.0, 1e-3, 260, 41, 10.0, 2000.0
    delay = 1.5 / f0
    c = n // 2
    s, x0, r = (8, c, c), (c + 6, c, c), (8, c, c + 10)
    fl = lambda p: (p[0] * n + p[1]) * n + p[2]
    w = _homog_workload(3, n, 10, dx, dt, nt, 8, f0, delay, fl(s), [fl(r)], v=v)
    dm = np.zeros((2, n, n, n))
    a = 1.0
    dm[0][x0] = a / 2
    dm[1][x0] = a / 2
    d = oracle.born(w, dm)[0]
    t = (np.arange(nt) + 1) * dt
    r1 = np.linalg.norm(np.subtract(x0, s)) * dx
    r2 = np.linalg.norm(np.subtract(r, x0)) * dx
    ref = analytic.born3d_kappa_point(r1, r2, t, v, f0, delay + dt / 2, a, dx ** 3)
    err = np.linalg.norm(d - ref) / np.linalg.norm(ref)
    assert err < 1.2e-2, err


@pytest.mark.parametrize("kind", ["kappa_only", "rho_only", "both"])
@pytest.mark.parametrize("ndim,order", [(2, 4), (2, 8), (3, 4)])
def test_linearisation(kind, ndim, order):
    """F(m0 + eps dm) - F(m0) - eps L dm = O(eps^2), with the perturbed model
    built from the definitions ln rho = ln Ip - ln Vp, ln kappa = ln Ip + ln Vp
    (Sec. 2): v -> v e^{eps dm1}, rho -> rho e^{eps (dm2 - dm1)}."""
    if ndim == 2:
        w = li.small_case(nz=22, nx=26, nt=140, order=order, npml=6, nshot=2, seed=5)
    else:
        w = li.small_case(ndim=3, nz=10, ny=9, nx=11, nt=60, order=order, npml=4, nshot=1, seed=6)
    dm = w.dm.copy()
    if kind == "kappa_only":
        dm[0] = dm[1]
    elif kind == "rho_only":
        dm[0] = -dm[1]
    vmax = float(np.max(w.vp))
    F0 = oracle.model(w, vmax=vmax)
    Ldm = oracle.born(w, dm, vmax=vmax)
    errs = []
    for eps in (1e-2, 1e-3):
        vp = w.vp * np.exp(eps * dm[0])
        rho = w.rho * np.exp(eps * (dm[1] - dm[0]))
        F1 = oracle.model(w, vp=vp, rho=rho, vmax=vmax)
        errs.append(np.linalg.norm(F1 - F0 - eps * Ldm) / np.linalg.norm(eps * Ldm))
    assert errs[1] < 5e-3, errs
    assert 8.0 < errs[0] / errs[1] < 12.5, errs


# --------------------------------------------------------- transposition

@pytest.mark.parametrize("ndim,order", [(2, 4), (2, 8), (3, 4), (3, 8)])
def test_dot_product(ndim, order):
    """<L m, d> = <m, L^T d> to 1e-12 relative on random m, d (App. A, as an
    exact discrete transpose), with CPML active."""
    rng = np.random.default_rng(100 + ndim * 10 + order)
    if ndim == 2:
        w = li.small_case(nz=20, nx=24, nt=120, order=order, npml=8, nshot=3, seed=order)
    else:
        w = li.small_case(ndim=3, nz=10, ny=9, nx=12, nt=50, order=order, npml=5, nshot=2,
                          seed=order)
    m = rng.standard_normal((2,) + w.shape)
    d = rng.standard_normal((w.geom.nrec_total, w.nt))
    a = float(np.vdot(oracle.born(w, m), d))
    b = float(np.vdot(m, oracle.adjoint(w, d)))
    assert abs(a - b) / max(abs(a), abs(b)) < 1e-12, (a, b)


def _explicit(w):
    n2 = 2 * w.nint
    nd = w.geom.nrec_total * w.nt
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
    return L, LT


def test_explicit_matrices_tiny():
    """Brute force on a tiny grid: the matrix of L^T built column by column
    from unit data vectors equals the transpose of the matrix of L built from
    unit model vectors."""
    w = li.small_case(nz=5, nx=6, nt=18, order=4, npml=3, nshot=1, seed=3, nrec=3)
    L, LT = _explicit(w)
    scale = np.abs(L).max()
    assert scale > 0
    np.testing.assert_allclose(LT, L.T, rtol=0, atol=1e-12 * scale)


def test_chain_rule_against_raw_gradients():
    """Sec. 3: g_Ip = g_rho + g_kappa, g_Vp = g_kappa - g_rho; and L of
    dm = (a, a) (pure dln kappa) equals the kappa part of L (checked via
    <L dm, d> = <dm, g>)."""
    w = li.small_case(nz=16, nx=18, nt=90, order=4, npml=5, nshot=2, seed=9)
    rng = np.random.default_rng(7)
    d = rng.standard_normal((w.geom.nrec_total, w.nt))
    g, graw = oracle.adjoint(w, d, raw=True)
    np.testing.assert_allclose(g[0] + g[1], 2 * graw[0], rtol=1e-13, atol=1e-13 * np.abs(g).max())
    np.testing.assert_allclose(g[1] - g[0], 2 * graw[1], rtol=1e-13, atol=1e-13 * np.abs(g).max())
    a = rng.standard_normal(w.shape)
    dm = np.stack([a, a])     # dln kappa = 2a, dln rho = 0
    lhs = float(np.vdot(oracle.born(w, dm), d))
    rhs = float(np.vdot(2 * a, graw[0]))
    assert abs(lhs - rhs) < 1e-12 * max(abs(lhs), abs(rhs))


# ---------------------------------------------------- CG, PSF, pseudo-Hessian

def _ls_case():
    w = li.small_case(nz=4, nx=5, nt=40, order=4, npml=3, nshot=2, seed=21, nrec=1)
    nint = w.nint
    # receivers at every interior node of each shot
    recs = np.arange(nint, dtype=np.int32)
    w.geom = Geometry(w.geom.src_idx, np.array([0, nint, 2 * nint], np.int32),
                      np.concatenate([recs, recs]))
    return w


def test_cgls_matches_dense_least_squares():
    """After more iterations than unknowns, CGNR on the oracle operators equals
    the dense least-squares solution of the explicit L (numpy lstsq), and the
    residual norm never increases (Sec. 3, CGNR)."""
    w = _ls_case()
    L, _ = _explicit_L_only(w)
    rng = np.random.default_rng(5)
    d = rng.standard_normal((w.geom.nrec_total, w.nt))
    x_ls = np.linalg.lstsq(L, d.ravel(), rcond=None)[0]
    x, mis = oracle.cgls(lambda m: oracle.born(w, m), lambda dd: oracle.adjoint(w, dd), d,
                         np.zeros((2,) + w.shape), 120)
    assert np.all(np.diff(mis) <= 1e-12)
    np.testing.assert_allclose(x.ravel(), x_ls, rtol=0, atol=1e-7 * np.abs(x_ls).max())
    # preconditioned variant converges to the same least-squares solution
    M = np.abs(rng.standard_normal((2,) + w.shape)) + 0.5
    xp, _ = oracle.cgls(lambda m: oracle.born(w, m), lambda dd: oracle.adjoint(w, dd), d,
                        np.zeros((2,) + w.shape), 120, precond=M)
    np.testing.assert_allclose(xp.ravel(), x_ls, rtol=0, atol=1e-7 * np.abs(x_ls).max())


def _explicit_L_only(w):
    n2 = 2 * w.nint
    L = np.zeros((w.geom.nrec_total * w.nt, n2))
    for j in range(n2):
        e = np.zeros(n2)
        e[j] = 1.0
        L[:, j] = oracle.born(w, e.reshape((2,) + w.shape)).ravel()
    return L, None


def test_cgls_param_mask_monoparameter():
    """With param_mask = 2 only dln Ip is updated and the result equals the
    least-squares solution over the Ip columns alone (the mono-parameter
    inversion of Sec. 5)."""
    w = _ls_case()
    L, _ = _explicit_L_only(w)
    rng = np.random.default_rng(6)
    d = rng.standard_normal((w.geom.nrec_total, w.nt))
    nint = w.nint
    x_ls = np.linalg.lstsq(L[:, nint:], d.ravel(), rcond=None)[0]
    x, _ = oracle.cgls(lambda m: oracle.born(w, m), lambda dd: oracle.adjoint(w, dd), d,
                       np.zeros((2,) + w.shape), 80, param_mask=2)
    assert np.all(x[0] == 0.0)
    np.testing.assert_allclose(x[1].ravel(), x_ls, rtol=0, atol=1e-7 * np.abs(x_ls).max())


def test_psf_is_sum_of_hessian_columns():
    """App. D: the PSF image of a spike comb is the sum of the Hessian columns
    L^T L e_j of its spikes, built from the explicit L."""
    w = li.small_case(nz=6, nx=6, nt=30, order=4, npml=3, nshot=2, seed=8, nrec=4)
    L, _ = _explicit_L_only(w)
    H = L.T @ L
    for param in (0, 1):
        cmb = oracle.comb(w.shape, 3, param)
        assert cmb.sum() == 4.0
        got = oracle.psf(w, param, 3).ravel()
        np.testing.assert_allclose(got, H @ cmb.ravel(), rtol=0, atol=1e-12 * np.abs(H).max())


def test_remigration_is_symmetric_and_positive():
    """App. D/E: H = L^T L is symmetric and positive semi-definite, so the
    remigration satisfies <H x, y> = <x, H y> and <H x, x> = |L x|^2 >= 0
    (2D and 3D, CPML active)."""
    for w in (li.small_case(nz=16, nx=20, nt=120, order=8, npml=6, nshot=2, seed=31, nrec=10),
              li.small_case(ndim=3, nz=8, ny=9, nx=10, nt=50, order=4, npml=4, nshot=1, seed=32, nrec=6)):
        rng = np.random.default_rng(7)
        x = rng.standard_normal((2,) + w.shape)
        y = rng.standard_normal((2,) + w.shape)
        hx = oracle.remigrate(w, x)
        hy = oracle.remigrate(w, y)
        a, b = float(np.vdot(hx, y)), float(np.vdot(x, hy))
        assert abs(a - b) <= 1e-12 * max(abs(a), abs(b))
        lx = oracle.born(w, x)
        assert abs(float(np.vdot(hx, x)) - float(np.vdot(lx, lx))) <= 1e-12 * float(np.vdot(lx, lx))


def test_pseudo_hessian_plane_wave():
    """App. B in nondimensional units (c = rho = 1): for a plane wave
    rho^2 |dv/dt|^2 = |grad p|^2 = |dp/dt|^2 = kappa^2 (div v)^2, so the
    pseudo-Hessian at a node is twice the time integral of (dp/dt)^2, computed
    here from the recorded pressure; also H_VpVp = H_IpIp by construction."""
    nz, nx = 80, 200
    vp = np.ones((nz, nx))
    rho = np.ones((nz, nx))
    dx, dt, f0, nt = 1.0, 0.25, 0.04, 600
    zs, zr = 20, 45
    geom = Geometry(np.array([zs * nx + nx // 2], np.int32), np.array([0, 1], np.int32),
                    np.array([zr * nx + nx // 2], np.int32))
    w = Workload("ph", 2, nz, 1, nx, dx, dx, dx, dt, nt, 8, 20, f0, vp, rho,
                 np.zeros((2, nz, nx)), li.ricker(nt, dt, f0, 1.5 / f0), geom)
    line = np.array([zs * nx + x for x in range(nx)], np.int32)
    sp = np.array([0, nx], np.int32)
    h = oracle.pseudo_hessian(w, src_ptr=sp, src_idx=line)
    p = oracle.model(w, src_ptr=sp, src_idx=line)[0]
    dp = np.diff(np.concatenate([[0.0], p])) / dt
    e_kappa = dt * np.sum(dp ** 2)
    ratio = h[zr, nx // 2] / e_kappa
    assert abs(ratio - 2.0) < 0.03, ratio
    assert np.all(h >= 0)
