"""FP64 CPU oracle for the LSRTM operator pair.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers. The product library
never imports this package and shares no code with it; inputs come from the
separate ``lsrtm_inputs`` module.

Layers:
  * ``lsrtm_oracle.c`` (compiled with gcc, FP64, no FMA contraction): the
    discrete background/nonlinear modelling of Eq. (1), Born modelling of
    Eq. (scattereqln), its exact transpose with the chain rule of Sec. 3 and
    the pseudo-Hessian of App. B.
  * this module: ctypes marshalling plus textbook FP64 numpy routines built on
    those operators: CGLS/CGNR and its diagonally preconditioned variant
    (Sec. 3), the spike comb and PSF / remigration probes (App. D).
  * ``deblur.py``: the nonstationary 11 x 11 deblurring filters of App. E
    (FP64 normal equations per comb window, bilinear valence blending).
  * ``psf_hessian.py``: the interpolated PSF Hessian of App. D and its
    image-domain CGNR.
  * ``data.py``: the muted data residuals of Sec. 4 (direct-wave and
    far-offset mutes of observed minus background data).

Pinned by the ``-m "not gpu"`` tests against: textbook staggered FD
coefficients, the 2D and 3D homogeneous Green's functions, the normal
incidence reflection coefficient (Z2-Z1)/(Z2+Z1), the 3D Born point-scatterer
closed form, the linearisation test against nonlinear modelling, the dot
product test, explicit matrices on tiny grids and dense least squares for CG.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
import sysconfig

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lsrtm_oracle.c")
_SO = os.path.join(_HERE, "_build", "liblsrtm_oracle.so")
_LIB = None


class Cfg(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int), ("nz", ctypes.c_int), ("ny", ctypes.c_int), ("nx", ctypes.c_int),
        ("npml", ctypes.c_int), ("order", ctypes.c_int), ("nt", ctypes.c_int),
        ("dz", ctypes.c_double), ("dy", ctypes.c_double), ("dx", ctypes.c_double),
        ("dt", ctypes.c_double), ("f0", ctypes.c_double), ("vmax", ctypes.c_double),
        ("free_surface", ctypes.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, -ffp-contract=off so x86 and Arm
    give the same rounding). Returns the path of the shared library."""
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
           "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _LIB
    if _LIB is None:
        build()
        L = ctypes.CDLL(_SO)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        cp = ctypes.POINTER(Cfg)
        L.orc_fd_coeffs.argtypes = [ctypes.c_int, dp]
        L.orc_model.argtypes = [cp, dp, dp, dp, ctypes.c_int, ctypes.c_int, ip, ip, ip, ip, dp]
        L.orc_born.argtypes = [cp, dp, dp, dp, ctypes.c_int, ctypes.c_int, ip, ip, ip, ip, dp, dp]
        L.orc_adjoint.argtypes = [cp, dp, dp, dp, ctypes.c_int, ctypes.c_int, ip, ip, ip, ip,
                                  dp, dp, dp]
        L.orc_pseudo_hessian.argtypes = [cp, dp, dp, dp, ctypes.c_int, ctypes.c_int, ip, ip, dp]
        L.orc_snapshot.argtypes = [cp, dp, dp, dp, ip, ip, ctypes.c_int, dp]
        L.orc_num_threads.argtypes = []
        _LIB = L
    return _LIB


def _d(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def num_threads() -> int:
    return int(lib().orc_num_threads())


def fd_coeffs(order: int) -> np.ndarray:
    c = np.zeros(4)
    if lib().orc_fd_coeffs(order, _d(c)):
        raise ValueError(f"unsupported order {order}")
    return c[: order // 2].copy()


def cfg_of(w, nt=None, vmax=None) -> Cfg:
    """Oracle configuration for a workload. The CPML damping uses the maximum
    background velocity unless `vmax` is given."""
    return Cfg(w.ndim, w.nz, w.ny, w.nx, w.npml, w.order, int(w.nt if nt is None else nt),
               w.dz, w.dy, w.dx, w.dt, w.f0,
               float(np.max(w.vp) if vmax is None else vmax),
               int(bool(getattr(w, "free_surface", False))))


def _src_csr(geom):
    n = geom.nshot
    return np.arange(n + 1, dtype=np.int32), _i32(geom.src_idx)


class _Args:
    def __init__(self, w, vp=None, rho=None, geom=None, wavelet=None, nt=None, vmax=None):
        self.w = w
        self.cfg = cfg_of(w, nt=nt, vmax=vmax)
        self.vp = _f64(w.vp if vp is None else vp)
        self.rho = _f64(w.rho if rho is None else rho)
        self.geom = w.geom if geom is None else geom
        wav = w.wavelet if wavelet is None else wavelet
        self.wav = _f64(wav)
        self.per_shot = 1 if self.wav.ndim == 2 else 0
        self.sp, self.si = _src_csr(self.geom)
        self.rp = _i32(self.geom.rec_ptr)
        self.ri = _i32(self.geom.rec_idx)
        self.nt = self.cfg.nt

    def common(self):
        return (ctypes.byref(self.cfg), _d(self.vp), _d(self.rho), _d(self.wav), self.per_shot,
                self.geom.nshot, _i(self.sp), _i(self.si), _i(self.rp), _i(self.ri))


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def model(w, vp=None, rho=None, geom=None, wavelet=None, nt=None, vmax=None,
          src_ptr=None, src_idx=None) -> np.ndarray:
    """Nonlinear modelling (Eq. 1): pressure records [nrec_total, nt]. A custom
    source list (CSR `src_ptr`, `src_idx`) overrides the one-source geometry;
    shots with aperture windows are modelled on their windows' sub-models."""
    g = w.geom if geom is None else geom
    if src_ptr is None and wavelet is None and windowed(g):
        return _model_windowed(w, vp, rho, g, nt, vmax)
    a = _Args(w, vp, rho, geom, wavelet, nt, vmax)
    d = np.zeros((a.geom.nrec_total, a.nt))
    args = list(a.common())
    if src_ptr is not None:
        sp, si = _i32(src_ptr), _i32(src_idx)
        args[6], args[7] = _i(sp), _i(si)
    _check(lib().orc_model(*args, _d(d)), "model")
    return d


def born(w, dm, vp=None, rho=None, geom=None, nt=None, vmax=None) -> np.ndarray:
    """d = L dm; dm [2, *shape] = (dln Vp, dln Ip); d [nrec_total, nt]."""
    geom = w.geom if geom is None else geom
    if windowed(geom):
        return _born_windowed(w, dm, vp, rho, geom, nt, vmax)
    a = _Args(w, vp, rho, geom, None, nt, vmax)
    dm = _f64(dm).reshape(2, -1)
    d = np.zeros((a.geom.nrec_total, a.nt))
    _check(lib().orc_born(*a.common(), _d(dm), _d(d)), "born")
    return d


def adjoint(w, d, vp=None, rho=None, geom=None, nt=None, vmax=None, raw=False):
    """g = L^T d as [2, *shape] (dln Vp, dln Ip). With raw=True also returns
    (g_kappa, g_rho) before the chain rule."""
    geom = w.geom if geom is None else geom
    if windowed(geom):
        if raw:
            raise ValueError("raw images are not provided for windowed geometries")
        return _adjoint_windowed(w, d, vp, rho, geom, nt, vmax)
    a = _Args(w, vp, rho, geom, None, nt, vmax)
    d = _f64(d).reshape(a.geom.nrec_total, a.nt)
    g = np.zeros((2, w.nint))
    gr = np.zeros((2, w.nint))
    _check(lib().orc_adjoint(*a.common(), _d(d), _d(g), _d(gr)), "adjoint")
    shape = (2,) + tuple(w.shape)
    if raw:
        return g.reshape(shape), gr.reshape(shape)
    return g.reshape(shape)


# ---------------------------------------------------------------------------
# Per-shot aperture windows. A shot with window [x0, x0 + nx_w) of interior
# columns is modelled on the sub-model vp[..., x0:x0+nx_w] (and rho, dm),
# padded with CPML and edge replication of that sub-model exactly as a full
# model is; its records are that sub-problem's records and its image is added
# into the window's columns. The CPML damping keeps the full model's
# maximum velocity. Source and receivers must lie inside the window.


def windowed(geom) -> bool:
    return geom is not None and getattr(geom, "win_x0", None) is not None


def _window_case(w, geom, s, vp, rho, vmax):
    import dataclasses
    x0 = int(geom.win_x0[s])
    nxw = int(geom.win_nx[s])
    if x0 < 0 or nxw < 1 or x0 + nxw > w.nx:
        raise ValueError(f"shot {s}: window outside the model")
    vp = w.vp if vp is None else vp
    rho = w.rho if rho is None else rho

    def local(k):
        k = np.asarray(k, np.int64)
        ix = k % w.nx
        rest = k // w.nx
        if np.any(ix < x0) or np.any(ix >= x0 + nxw):
            raise ValueError(f"shot {s}: source or receiver outside its window")
        return (rest * nxw + (ix - x0)).astype(np.int32)

    r = geom.rec_idx[geom.rec_ptr[s]:geom.rec_ptr[s + 1]]
    g1 = type(geom)(src_idx=local([geom.src_idx[s]]), rec_ptr=np.array([0, r.size], np.int32),
                    rec_idx=local(r))
    wav = w.wavelet if np.ndim(w.wavelet) == 1 else np.asarray(w.wavelet)[s]
    sub = dataclasses.replace(w, nx=nxw, vp=np.ascontiguousarray(vp[..., x0:x0 + nxw]),
                              rho=np.ascontiguousarray(rho[..., x0:x0 + nxw]),
                              dm=None, wavelet=wav, geom=g1)
    vmax = float(np.max(vp)) if vmax is None else vmax
    return sub, x0, nxw, vmax


def _born_windowed(w, dm, vp, rho, geom, nt, vmax):
    dm = _f64(dm).reshape((2,) + tuple(w.shape))
    ntt = int(w.nt if nt is None else nt)
    d = np.zeros((geom.nrec_total, ntt))
    for s in range(geom.nshot):
        sub, x0, nxw, vm = _window_case(w, geom, s, vp, rho, vmax)
        d[geom.rec_ptr[s]:geom.rec_ptr[s + 1]] = born(
            sub, np.ascontiguousarray(dm[..., x0:x0 + nxw]), nt=nt, vmax=vm)
    return d


def _model_windowed(w, vp, rho, geom, nt, vmax):
    ntt = int(w.nt if nt is None else nt)
    d = np.zeros((geom.nrec_total, ntt))
    for s in range(geom.nshot):
        sub, x0, nxw, vm = _window_case(w, geom, s, vp, rho, vmax)
        d[geom.rec_ptr[s]:geom.rec_ptr[s + 1]] = model(sub, nt=nt, vmax=vm)
    return d


def _adjoint_windowed(w, d, vp, rho, geom, nt, vmax):
    ntt = int(w.nt if nt is None else nt)
    d = _f64(d).reshape(geom.nrec_total, ntt)
    g = np.zeros((2,) + tuple(w.shape))
    for s in range(geom.nshot):
        sub, x0, nxw, vm = _window_case(w, geom, s, vp, rho, vmax)
        g[..., x0:x0 + nxw] += adjoint(sub, d[geom.rec_ptr[s]:geom.rec_ptr[s + 1]], nt=nt, vmax=vm)
    return g


def pseudo_hessian(w, vp=None, rho=None, geom=None, nt=None, vmax=None,
                   src_ptr=None, src_idx=None) -> np.ndarray:
    """Pseudo-Hessian diagonal (App. B), interior shape; serves both planes.
    A custom source list (CSR) may replace the one-source geometry."""
    g0 = w.geom if geom is None else geom
    if src_ptr is None and windowed(g0):
        h = np.zeros(tuple(w.shape))
        for s in range(g0.nshot):
            sub, x0, nxw, vm = _window_case(w, g0, s, vp, rho, vmax)
            h[..., x0:x0 + nxw] += pseudo_hessian(sub, nt=nt, vmax=vm)
        return h
    a = _Args(w, vp, rho, geom, None, nt, vmax)
    h = np.zeros(w.nint)
    args = list(a.common()[:8])
    if src_ptr is not None:
        sp, si = _i32(src_ptr), _i32(src_idx)
        args[5] = len(sp) - 1
        args[6], args[7] = _i(sp), _i(si)
    _check(lib().orc_pseudo_hessian(*args, _d(h)), "pseudo_hessian")
    return h.reshape(w.shape)


def snapshot(w, nsnap, src_ptr=None, src_idx=None, vp=None, rho=None, vmax=None):
    """Padded pressure field p^{nsnap} of shot 0 (or of a custom source list)."""
    a = _Args(w, vp, rho, None, None, None, vmax)
    sp = a.sp if src_ptr is None else _i32(src_ptr)
    si = a.si if src_idx is None else _i32(src_idx)
    npad = [w.nz + 2 * w.npml, (w.ny + 2 * w.npml) if w.ndim == 3 else 1, w.nx + 2 * w.npml]
    p = np.zeros(int(np.prod(npad)))
    _check(lib().orc_snapshot(ctypes.byref(a.cfg), _d(a.vp), _d(a.rho), _d(a.wav), _i(sp),
                              _i(si), int(nsnap), _d(p)), "snapshot")
    return p.reshape(npad if w.ndim == 3 else (npad[0], npad[2]))


# ---------------------------------------------------------------------------
# Krylov solver and probes (FP64 numpy on top of the operators)
# ---------------------------------------------------------------------------

def _mask(param_mask, shape):
    m = np.zeros((2,) + tuple(shape))
    if param_mask & 1:
        m[0] = 1.0
    if param_mask & 2:
        m[1] = 1.0
    return m


def cgls(apply_L, apply_LT, d, x0, niter, precond=None, param_mask=3):
    """CGNR (CGLS form) on min ||L x - d||^2 with x restricted to the planes in
    `param_mask` (1 = dln Vp, 2 = dln Ip). With `precond` (a diagonal M given
    as its inverse, same shape as x) this is the preconditioned CGNR of
    Sec. 3. Returns x and the normalised misfits ||d - L x_k|| / ||d||,
    k = 0..niter."""
    P = _mask(param_mask, x0.shape[1:])
    Minv = P if precond is None else P * precond
    x = x0 * P
    r = d - apply_L(x)
    s = apply_LT(r) * P
    z = s * Minv
    p = z.copy()
    gamma = float(np.vdot(s, z))
    dn = float(np.linalg.norm(d))
    mis = [float(np.linalg.norm(r)) / dn]
    for _ in range(niter):
        q = apply_L(p)
        qq = float(np.vdot(q, q))
        if qq == 0.0 or gamma == 0.0:
            mis.append(mis[-1])
            continue
        alpha = gamma / qq
        x = x + alpha * p
        r = r - alpha * q
        s = apply_LT(r) * P
        z = s * Minv
        gnew = float(np.vdot(s, z))
        beta = gnew / gamma
        p = z + beta * p
        gamma = gnew
        mis.append(float(np.linalg.norm(r)) / dn)
    return x, np.asarray(mis)


def pcg_diag_from_hessian(h, eps=1e-3):
    """Inverse of the diagonal preconditioner M = H + eps * max(H) (App. B),
    applied to both parameter planes."""
    m = h + eps * float(np.max(h))
    inv = 1.0 / m
    return np.stack([inv, inv])


def lsrtm_cg(w, d, niter, precond=False, param_mask=3, x0=None):
    """Data-domain LSRTM by CGNR / PCGNR with the oracle operators."""
    x0 = np.zeros((2,) + tuple(w.shape)) if x0 is None else np.asarray(x0, np.float64)
    M = pcg_diag_from_hessian(pseudo_hessian(w)) if precond else None
    return cgls(lambda m: born(w, m), lambda dd: adjoint(w, dd), np.asarray(d, np.float64),
                x0, niter, precond=M, param_mask=param_mask)


def comb(shape, spacing, param):
    """Spike comb of App. D: unit spikes every `spacing` cells along every axis
    starting at spacing//2, in parameter plane `param` (0 = Vp, 1 = Ip)."""
    out = np.zeros((2,) + tuple(shape))
    sl = tuple(slice(spacing // 2, None, spacing) for _ in shape)
    out[(param,) + sl] = 1.0
    return out


def psf(w, param, spacing):
    """PSF image L^T L comb (App. D)."""
    return adjoint(w, born(w, comb(w.shape, spacing, param)))


def remigrate(w, m):
    """Remigrated image m'' = L^T L m (App. E)."""
    return adjoint(w, born(w, m))
