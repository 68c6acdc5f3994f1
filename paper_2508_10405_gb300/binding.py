"""Thin ctypes binding of the C ABI in include/lsrtm.h.

Argument marshalling only: every step of the operators runs in the CUDA
library. Loading fails loudly if liblsrtm.so is missing or cannot be loaded;
there is no CPU fallback.

Arrays may be CUDA tensors (float32, contiguous) or host numpy / torch CPU
arrays; results come back as CUDA tensors unless host output was requested.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SO_PATH = os.path.join(_HERE, "_lib", "liblsrtm.so")

LSRTM_OK = 0
STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_CFL", 3: "ERR_GEOMETRY", 4: "ERR_OOM",
          5: "ERR_NONFINITE", 6: "ERR_CUDA", 7: "ERR_STATE"}
BAND_FP32, BAND_BF16, BAND_FP16 = 0, 1, 2
RECON_BOUNDARY, RECON_CHECKPOINT, RECON_AUTO = 0, 1, 2
PLAN_BATCHED, PLAN_PLAIN = 0, 1

# Every symbol include/lsrtm.h declares.
EXPORTS = ["lsrtm_create", "lsrtm_born", "lsrtm_adjoint", "lsrtm_psf", "lsrtm_remigrate",
           "lsrtm_cg_solve", "lsrtm_cg_begin", "lsrtm_cg_iterate", "lsrtm_cg_result",
           "lsrtm_timing_enable", "lsrtm_timing_read", "lsrtm_set_stream",
           "lsrtm_workspace_bytes", "lsrtm_kernel_launches", "lsrtm_destroy", "lsrtm_last_error",
           "lsrtm_born_static", "lsrtm_reconstruction", "lsrtm_deblur", "lsrtm_autotune",
           "lsrtm_psf_hessian", "lsrtm_psf_cg", "lsrtm_model", "lsrtm_mute_residual",
           "lsrtm_deblur_wiener", "lsrtm_cg_get_state", "lsrtm_cg_set_state", "lsrtm_synchronize"]


class LsrtmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Config(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int), ("nz", ctypes.c_int), ("ny", ctypes.c_int), ("nx", ctypes.c_int),
        ("dz", ctypes.c_double), ("dy", ctypes.c_double), ("dx", ctypes.c_double),
        ("dt", ctypes.c_double), ("nt", ctypes.c_int), ("fd_order", ctypes.c_int),
        ("npml", ctypes.c_int), ("f0", ctypes.c_double), ("pml_vmax", ctypes.c_double),
        ("band_precision", ctypes.c_int), ("hbm_budget_bytes", ctypes.c_size_t),
        ("recon_mode", ctypes.c_int), ("plan", ctypes.c_int), ("shots_per_batch", ctypes.c_int),
        ("wavelet_per_shot", ctypes.c_int), ("checkpoint_interval", ctypes.c_int),
        ("free_surface", ctypes.c_int), ("guard_interval", ctypes.c_int),
        ("checkpoint_precision", ctypes.c_int),
    ]


class Timings(ctypes.Structure):
    _fields_ = [("born_ms", ctypes.c_double), ("background_ms", ctypes.c_double),
                ("adjoint_ms", ctypes.c_double), ("born_launches", ctypes.c_longlong),
                ("background_launches", ctypes.c_longlong), ("adjoint_launches", ctypes.c_longlong),
                ("born_cells", ctypes.c_double), ("background_cells", ctypes.c_double),
                ("adjoint_cells", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class GeometryC(ctypes.Structure):
    _fields_ = [("nshot", ctypes.c_int), ("src_idx", ctypes.POINTER(ctypes.c_int)),
                ("rec_ptr", ctypes.POINTER(ctypes.c_int)), ("rec_idx", ctypes.POINTER(ctypes.c_int)),
                ("win_x0", ctypes.POINTER(ctypes.c_int)), ("win_nx", ctypes.POINTER(ctypes.c_int))]


_LIB = None


def load_library(path: str | None = None):
    """Loads liblsrtm.so (building it first if it is absent and nvcc exists)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = path or SO_PATH
    if not os.path.exists(path):
        from . import build as _build
        _build.build()
    L = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    L.lsrtm_create.argtypes = [ctypes.POINTER(Config), vp, vp, vp, ctypes.POINTER(GeometryC), vp,
                               ctypes.POINTER(vp)]
    L.lsrtm_born.argtypes = [vp, vp, vp]
    L.lsrtm_adjoint.argtypes = [vp, vp, vp, vp]
    L.lsrtm_psf.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp]
    L.lsrtm_remigrate.argtypes = [vp, vp, vp]
    L.lsrtm_cg_solve.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 ctypes.POINTER(ctypes.c_double)]
    L.lsrtm_cg_begin.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_int]
    L.lsrtm_cg_iterate.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    L.lsrtm_cg_result.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_double)]
    L.lsrtm_timing_enable.argtypes = [vp, ctypes.c_int]
    L.lsrtm_timing_read.argtypes = [vp, ctypes.POINTER(Timings), ctypes.c_int]
    L.lsrtm_set_stream.argtypes = [vp, vp]
    L.lsrtm_synchronize.argtypes = [vp]
    L.lsrtm_born_static.argtypes = [ctypes.POINTER(Config), vp, vp, vp, ctypes.POINTER(GeometryC), vp, vp, vp]
    ip = ctypes.POINTER(ctypes.c_int)
    L.lsrtm_reconstruction.argtypes = [vp, ip, ip, ip]
    L.lsrtm_autotune.argtypes = [vp, ctypes.c_int, ip, ctypes.POINTER(ctypes.c_double), ip]
    L.lsrtm_deblur.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_double, vp, vp]
    L.lsrtm_cg_get_state.argtypes = [vp, vp, vp, vp, ctypes.POINTER(ctypes.c_double), ip]
    L.lsrtm_cg_set_state.argtypes = [vp, vp, vp, vp, ctypes.POINTER(ctypes.c_double), ctypes.c_int]
    L.lsrtm_deblur_wiener.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_double, vp]
    L.lsrtm_model.argtypes = [vp, vp]
    L.lsrtm_mute_residual.argtypes = [vp, vp, vp] + [ctypes.c_double] * 5 + [vp]
    L.lsrtm_psf_hessian.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp]
    L.lsrtm_psf_cg.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp, ctypes.c_int,
                               ctypes.POINTER(ctypes.c_double)]
    L.lsrtm_workspace_bytes.argtypes = [vp]
    L.lsrtm_workspace_bytes.restype = ctypes.c_size_t
    L.lsrtm_kernel_launches.argtypes = [vp]
    L.lsrtm_kernel_launches.restype = ctypes.c_longlong
    L.lsrtm_destroy.argtypes = [vp]
    L.lsrtm_destroy.restype = None
    L.lsrtm_last_error.argtypes = []
    L.lsrtm_last_error.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("lsrtm_workspace_bytes", "lsrtm_kernel_launches", "lsrtm_destroy",
                        "lsrtm_last_error"):
            getattr(L, name).restype = ctypes.c_int
    _LIB = L
    return L


def _check(rc: int):
    if rc != LSRTM_OK:
        raise LsrtmError(rc, load_library().lsrtm_last_error().decode())


def _ptr(a):
    """Raw pointer of a torch tensor or numpy array (float32/int32, contiguous)."""
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("array must be contiguous")
        return ctypes.c_void_p(a.data_ptr())
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be contiguous")
    return ctypes.c_void_p(a.ctypes.data)


def _f32(a):
    if hasattr(a, "data_ptr"):
        import torch
        if a.dtype != torch.float32:
            raise TypeError("expected float32")
        return a.contiguous()
    return np.ascontiguousarray(a, dtype=np.float32)


class Lsrtm:
    """Operator handle: L (born), L^T (adjoint), PSF, remigration, CGNR.

    Parameters mirror lsrtm_config; `vp`, `rho` are [nz, (ny,) nx] arrays,
    `wavelet` [nt] (or [nshot, nt]), geometry = (src_idx, rec_ptr, rec_idx)
    flat interior indices. `stream` is a torch.cuda.Stream or raw handle
    (default: torch's current stream)."""

    def __init__(self, *, ndim, nz, nx, ny=1, dz, dx, dy=None, dt, nt, fd_order, npml, f0,
                 vp, rho, wavelet, src_idx, rec_ptr, rec_idx, win_x0=None, win_nx=None, pml_vmax=None,
                 band_precision=BAND_FP32, hbm_budget_bytes=0, recon_mode=RECON_AUTO,
                 plan=PLAN_BATCHED, shots_per_batch=0, checkpoint_interval=0, free_surface=False,
                 guard_interval=0, checkpoint_precision=BAND_FP32, stream=None):
        import torch
        self._lib = load_library()
        self._h = ctypes.c_void_p()
        vp = _f32(vp)
        rho = _f32(rho)
        wav = _f32(wavelet)
        if pml_vmax is None:
            pml_vmax = float(vp.max())
        self.cfg = Config(ndim, nz, ny if ndim == 3 else 1, nx, dz, dy or dx, dx, dt, nt,
                          fd_order, npml, f0, float(pml_vmax), band_precision,
                          int(hbm_budget_bytes), recon_mode, plan, shots_per_batch,
                          1 if np.ndim(wavelet) == 2 else 0, int(checkpoint_interval), int(bool(free_surface)),
                          int(guard_interval), int(checkpoint_precision))
        self._src = np.ascontiguousarray(src_idx, dtype=np.int32)
        self._rp = np.ascontiguousarray(rec_ptr, dtype=np.int32)
        self._ri = np.ascontiguousarray(rec_idx, dtype=np.int32)
        ip = ctypes.POINTER(ctypes.c_int)
        self._wx0 = None if win_x0 is None else np.ascontiguousarray(win_x0, dtype=np.int32)
        self._wnx = None if win_nx is None else np.ascontiguousarray(win_nx, dtype=np.int32)
        geo = GeometryC(len(self._src), self._src.ctypes.data_as(ip), self._rp.ctypes.data_as(ip),
                        self._ri.ctypes.data_as(ip),
                        None if self._wx0 is None else self._wx0.ctypes.data_as(ip),
                        None if self._wnx is None else self._wnx.ctypes.data_as(ip))
        self.nshot = len(self._src)
        self.nrec_total = int(self._rp[-1])
        self.nt = nt
        self.ndim = ndim
        self.shape = (nz, nx) if ndim == 2 else (nz, ny, nx)
        self.nint = int(np.prod(self.shape))
        self.device = torch.device("cuda", torch.cuda.current_device())
        self._stream = self._stream_handle(stream)
        _check(self._lib.lsrtm_create(ctypes.byref(self.cfg), _ptr(vp), _ptr(rho), _ptr(wav),
                                      ctypes.byref(geo), self._stream, ctypes.byref(self._h)))

    @staticmethod
    def _stream_handle(stream):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream()
        if hasattr(stream, "cuda_stream"):
            return ctypes.c_void_p(stream.cuda_stream)
        return ctypes.c_void_p(stream)

    @classmethod
    def from_workload(cls, w, **kw):
        """Handle for an lsrtm_inputs.Workload."""
        return cls(ndim=w.ndim, nz=w.nz, ny=w.ny, nx=w.nx, dz=w.dz, dy=w.dy, dx=w.dx, dt=w.dt,
                   nt=w.nt, fd_order=w.order, npml=w.npml, f0=w.f0, vp=w.vp, rho=w.rho,
                   wavelet=w.wavelet, src_idx=w.geom.src_idx, rec_ptr=w.geom.rec_ptr,
                   rec_idx=w.geom.rec_idx, win_x0=getattr(w.geom, "win_x0", None),
                   win_nx=getattr(w.geom, "win_nx", None),
                   **({"free_surface": getattr(w, "free_surface", False)} | kw))

    @property
    def model_shape(self) -> tuple:
        """Interior model grid, (nz, nx) or (nz, ny, nx)."""
        return self.shape

    # -- helpers
    def _empty(self, shape):
        import torch
        return torch.empty(shape, dtype=torch.float32, device=self.device)

    def _sync_stream(self):
        _check(self._lib.lsrtm_set_stream(self._h, self._stream_handle(None)))

    @property
    def handle(self):
        return self._h

    def synchronize(self):
        """Waits for the handle's queued work; raises LsrtmError if a kernel
        recorded a failure on the device."""
        _check(self._lib.lsrtm_synchronize(self._h))

    def workspace_bytes(self) -> int:
        return int(self._lib.lsrtm_workspace_bytes(self._h))

    def kernel_launches(self) -> int:
        return int(self._lib.lsrtm_kernel_launches(self._h))

    def autotune(self, steps=16) -> dict:
        """Times the 2D z-chunk candidates and keeps the fastest;
        {"tzc": chosen rows per chunk, "ms_per_step": {tzc: ms}}."""
        self._sync_stream()
        t, n = ctypes.c_int(), ctypes.c_int()
        ms = (ctypes.c_double * 32)()
        _check(self._lib.lsrtm_autotune(self._h, int(steps), ctypes.byref(t), ms, ctypes.byref(n)))
        return {"tzc": t.value, "ms_per_step": {int(ms[2 * i]): ms[2 * i + 1] for i in range(n.value)}}

    def reconstruction(self) -> dict:
        """{"mode": RECON_BOUNDARY | RECON_CHECKPOINT, "interval": K, "batch": shots per batch}."""
        m, k, b = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(self._lib.lsrtm_reconstruction(self._h, ctypes.byref(m), ctypes.byref(k), ctypes.byref(b)))
        return {"mode": m.value, "interval": k.value, "batch": b.value}

    # -- operators
    def born(self, dm, out=None):
        """d = L dm: dm [2, *shape] -> d [nrec_total, nt]."""
        self._sync_stream()
        dm = _f32(dm)
        out = self._empty((self.nrec_total, self.nt)) if out is None else out
        _check(self._lib.lsrtm_born(self._h, _ptr(dm), _ptr(out)))
        return out

    def adjoint(self, d, out=None, pseudo_hessian=False):
        """g = L^T d: d [nrec_total, nt] -> g [2, *shape] (and the pseudo-Hessian)."""
        self._sync_stream()
        d = _f32(d)
        out = self._empty((2,) + self.shape) if out is None else out
        ph = self._empty(self.shape) if pseudo_hessian else None
        _check(self._lib.lsrtm_adjoint(self._h, _ptr(d), _ptr(out),
                                       _ptr(ph) if ph is not None else None))
        return (out, ph) if pseudo_hessian else out

    def pseudo_hessian(self):
        """Pseudo-Hessian diagonal of App. B over this handle's shots,
        [*shape] (cached by the library once computed)."""
        import torch
        z = torch.zeros((self.nrec_total, self.nt), dtype=torch.float32, device=self.device)
        return self.adjoint(z, pseudo_hessian=True)[1]

    def psf(self, param, spacing, out=None):
        """PSF = L^T L comb (comb: unit spikes every `spacing` in plane `param`)."""
        self._sync_stream()
        out = self._empty((2,) + self.shape) if out is None else out
        _check(self._lib.lsrtm_psf(self._h, int(param), int(spacing), _ptr(out)))
        return out

    def remigrate(self, m, out=None):
        """m'' = L^T L m."""
        self._sync_stream()
        m = _f32(m)
        out = self._empty((2,) + self.shape) if out is None else out
        _check(self._lib.lsrtm_remigrate(self._h, _ptr(m), _ptr(out)))
        return out

    def deblur(self, m_rtm, m_remig, spacing=20, flen=11, eps=1e-3, return_filters=False):
        """Nonstationary deblurring filters (App. E): flen x flen filters per
        comb node from FP64 normal equations, blended image of m_rtm.
        Returns dm (and the filters [2, nkz, nkx, flen, flen] on request)."""
        self._sync_stream()
        a, b = _f32(m_rtm), _f32(m_remig)
        out = self._empty((2,) + self.shape)
        filt = None
        if return_filters:
            nk = [len(range(spacing // 2, n, spacing)) for n in self.shape]
            filt = self._empty((2, nk[0], nk[1], flen, flen))
        _check(self._lib.lsrtm_deblur(self._h, _ptr(a), _ptr(b), int(spacing), int(flen), float(eps),
                                      _ptr(out), None if filt is None else _ptr(filt)))
        return (out, filt) if return_filters else out

    def model(self, out=None):
        """Nonlinear modelling (Eq. 1) in the handle's own model: pressure
        records [nrec_total, nt]."""
        self._sync_stream()
        out = self._empty((self.nrec_total, self.nt)) if out is None else out
        _check(self._lib.lsrtm_model(self._h, _ptr(out)))
        return out

    def mute_residual(self, d_obs, d_syn, v_mute, t0, t_taper, o_max=0.0, o_taper=0.0, out=None):
        """Muted data residual (Sec. 4): the direct-wave mute after
        offset / v_mute + t0 (raised-cosine rise over t_taper) times the
        far-offset cut at o_max (rise over o_taper), applied to d_obs - d_syn
        (d_syn may be None)."""
        self._sync_stream()
        a = _f32(d_obs)
        b = None if d_syn is None else _f32(d_syn)
        out = self._empty((self.nrec_total, self.nt)) if out is None else out
        _check(self._lib.lsrtm_mute_residual(self._h, _ptr(a), None if b is None else _ptr(b), float(v_mute),
                                             float(t0), float(t_taper), float(o_max), float(o_taper), _ptr(out)))
        return out

    def psf_hessian(self, x, psf_vp, psf_ip, spacing=20, half=-1, transpose=False, param_mask=3, out=None):
        """y = P H P x (or P H^T P x) with the PSF Hessian interpolated on the
        fly from the PSF images of the combs in Vp and Ip (App. D); half < 0
        selects (spacing - 1) // 2. The PSF of a parameter outside param_mask
        may be None."""
        self._sync_stream()
        x = _f32(x)
        pv = None if psf_vp is None else _f32(psf_vp)
        pi = None if psf_ip is None else _f32(psf_ip)
        out = self._empty((2,) + self.shape) if out is None else out
        _check(self._lib.lsrtm_psf_hessian(self._h, None if pv is None else _ptr(pv),
                                           None if pi is None else _ptr(pi), int(spacing), int(half),
                                           int(param_mask), int(bool(transpose)), _ptr(x), _ptr(out)))
        return out

    def psf_cg(self, m_rtm, psf_vp, psf_ip, niter, spacing=20, half=-1, param_mask=3):
        """Image-domain CGNR on H^H H dm = H^H P m_rtm with the interpolated
        PSF Hessian (App. D); returns (dm, misfit history of length niter+1)."""
        self._sync_stream()
        m = _f32(m_rtm)
        pv = None if psf_vp is None else _f32(psf_vp)
        pi = None if psf_ip is None else _f32(psf_ip)
        out = self._empty((2,) + self.shape)
        mis = (ctypes.c_double * (niter + 1))()
        _check(self._lib.lsrtm_psf_cg(self._h, None if pv is None else _ptr(pv), None if pi is None else _ptr(pi),
                                      int(spacing), int(half), int(param_mask), _ptr(m), _ptr(out), int(niter),
                                      mis))
        return out, np.array(list(mis))

    def deblur_wiener(self, m_rtm, m_remig, spacing=20, eps=1e-3, out=None):
        """Nonstationary Wiener deblurring (App. E, Fourier form): per comb
        node a 2s x 2s block filtered by conj(F m'') F m_rtm / (|F m''|^2 +
        eps mean|F m''|^2), blended with the bilinear valence."""
        self._sync_stream()
        a, b = _f32(m_rtm), _f32(m_remig)
        out = self._empty((2,) + self.shape) if out is None else out
        _check(self._lib.lsrtm_deblur_wiener(self._h, _ptr(a), _ptr(b), int(spacing), float(eps), _ptr(out)))
        return out

    def cg_solve(self, d, niter, x0=None, precond=False, param_mask=3, log=None, m_true=None):
        """CGNR / PCGNR; returns (dm, misfit history of length niter+1).
        With `log` (a path, "-" for stderr or a file object; default: the
        LSRTM_PROFILE environment variable) the solve runs step-wise and
        writes one JSON line per iteration (cglog): misfit, relative model
        error against `m_true` if given, seconds, Gcell/s and GB/s."""
        import torch
        from . import cglog
        log = log if log is not None else cglog.env_log()
        if log is not None:
            return cglog.cg_solve_logged(self, d, niter, x0=x0, precond=precond, param_mask=param_mask,
                                         log=log, m_true=m_true)
        self._sync_stream()
        d = _f32(d)
        x = torch.zeros((2,) + self.shape, dtype=torch.float32, device=self.device) \
            if x0 is None else _f32(x0).clone()
        mis = (ctypes.c_double * (niter + 1))()
        _check(self._lib.lsrtm_cg_solve(self._h, _ptr(d), _ptr(x), int(niter), int(bool(precond)),
                                        int(param_mask), mis))
        return x, np.array(list(mis))

    def cg_begin(self, d, x0=None, precond=False, param_mask=3):
        """Starts a step-wise CGNR solve (r0 = d - L x0, s0 = L^T r0)."""
        self._sync_stream()
        d = _f32(d)
        self._cg_keep = (d, None if x0 is None else _f32(x0))
        _check(self._lib.lsrtm_cg_begin(self._h, _ptr(d),
                                        None if x0 is None else _ptr(self._cg_keep[1]),
                                        int(bool(precond)), int(param_mask)))

    def cg_get_state(self) -> dict:
        """State of the active step-wise CGNR solve as host numpy arrays:
        x, p [2, *shape], r [nrec_total, nt], scalars [gamma, <d,d>], iter."""
        self._sync_stream()
        x = np.empty((2,) + self.shape, np.float32)
        p = np.empty_like(x)
        r = np.empty((self.nrec_total, self.nt), np.float32)
        sc = (ctypes.c_double * 2)()
        it = ctypes.c_int()
        _check(self._lib.lsrtm_cg_get_state(self._h, _ptr(x), _ptr(p), _ptr(r), sc, ctypes.byref(it)))
        return {"x": x, "p": p, "r": r, "scalars": np.array(list(sc)), "iter": int(it.value)}

    def cg_set_state(self, state: dict):
        """Restores a state from cg_get_state after cg_begin with the same d,
        precond and param_mask; later cg_iterate calls continue bit for bit."""
        self._sync_stream()
        x = np.ascontiguousarray(state["x"], np.float32)
        p = np.ascontiguousarray(state["p"], np.float32)
        r = np.ascontiguousarray(state["r"], np.float32)
        sc = (ctypes.c_double * 2)(*[float(v) for v in state["scalars"]])
        _check(self._lib.lsrtm_cg_set_state(self._h, _ptr(x), _ptr(p), _ptr(r), sc, int(state["iter"])))

    def cg_iterate(self, niter=1, misfit=False):
        """Runs niter CGNR iterations; returns their misfits if misfit=True."""
        self._sync_stream()
        if misfit:
            mis = (ctypes.c_double * max(niter, 1))()
            _check(self._lib.lsrtm_cg_iterate(self._h, int(niter), mis))
            return np.array(list(mis))[:niter]
        _check(self._lib.lsrtm_cg_iterate(self._h, int(niter), None))
        return None

    def cg_result(self):
        """Current CGNR iterate [2, *shape] and the misfit of x0."""
        self._sync_stream()
        x = self._empty((2,) + self.shape)
        m0 = ctypes.c_double()
        _check(self._lib.lsrtm_cg_result(self._h, _ptr(x), ctypes.byref(m0)))
        return x, float(m0.value)

    def timing(self, enable=True):
        _check(self._lib.lsrtm_timing_enable(self._h, int(bool(enable))))

    def timings(self, reset=False) -> dict:
        t = Timings()
        _check(self._lib.lsrtm_timing_read(self._h, ctypes.byref(t), int(bool(reset))))
        return t.as_dict()

    def close(self):
        if self._h:
            self._lib.lsrtm_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def born_op():
    """torch.autograd.Function whose forward is L and backward is L^T, both
    in the CUDA library: BornOp.apply(dm, handle) -> d."""
    import torch

    class BornOp(torch.autograd.Function):
        @staticmethod
        def forward(ctx, dm, handle):
            ctx.handle = handle
            return handle.born(dm.detach())

        @staticmethod
        def backward(ctx, grad_d):
            return ctx.handle.adjoint(grad_d.contiguous()), None

    return BornOp
