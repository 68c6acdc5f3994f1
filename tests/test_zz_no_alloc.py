"""lsrtm_born_static: Born modelling for callers that cannot allocate device
memory (host applications that own the GPU memory pool and forbid foreign
allocations, real-time loops that must not allocate). It must give the same
records as lsrtm_born
(the handle-based entry point) within the parity tolerance, on consecutive
calls that share its fixed static workspace, and must refuse problems larger
than that workspace with a clear error.

This file is collected last on purpose: a failure here does not hide the
results of the other GPU tests in a run that stops at the first failure."""
import ctypes

import numpy as np
import pytest

import lsrtm_inputs as li

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 1e-4


def _static_call(lib, w, dm_dev, d_dev, dev=None):
    from paper_2508_10405_gb300.binding import Config, GeometryC
    cfg = Config(2, w.nz, 1, w.nx, w.dz, w.dy, w.dx, w.dt, w.nt, w.order, w.npml, w.f0,
                 float(np.max(w.vp)), 0, 0, 0, 0, 0, 0)
    src = np.ascontiguousarray(w.geom.src_idx, np.int32)
    rp = np.ascontiguousarray(w.geom.rec_ptr, np.int32)
    ri = np.ascontiguousarray(w.geom.rec_idx, np.int32)
    ip = ctypes.POINTER(ctypes.c_int)
    geo = GeometryC(len(src), src.ctypes.data_as(ip), rp.ctypes.data_as(ip), ri.ctypes.data_as(ip))
    if dev is None:
        dev = (torch.tensor(w.vp, dtype=torch.float32, device="cuda"),
               torch.tensor(w.rho, dtype=torch.float32, device="cuda"),
               torch.tensor(w.wavelet, dtype=torch.float32, device="cuda"))
    vp, rho, wav = dev
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.lsrtm_born_static(ctypes.byref(cfg), ctypes.c_void_p(vp.data_ptr()),
                               ctypes.c_void_p(rho.data_ptr()), ctypes.c_void_p(wav.data_ptr()),
                               ctypes.byref(geo), ctypes.c_void_p(dm_dev.data_ptr()),
                               ctypes.c_void_p(d_dev.data_ptr()), stream)
    torch.cuda.synchronize()
    return rc


def _rel(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_static_born_matches_handle_born_on_consecutive_calls():
    from paper_2508_10405_gb300 import Lsrtm, load_library
    lib = load_library()
    w = li.small_case(nz=46, nx=58, nt=240, order=8, npml=10, nshot=3, seed=91)
    h = Lsrtm.from_workload(w)
    dm = torch.tensor(w.dm, dtype=torch.float32, device="cuda")
    ref = h.born(dm)
    torch.cuda.synchronize()
    outs = [torch.full((w.geom.nrec_total, w.nt), float("nan"), dtype=torch.float32, device="cuda")
            for _ in range(2)]
    # the inputs of the calls exist before the first one, so the device's free
    # memory can only change if a call allocates
    vp = torch.tensor(w.vp, dtype=torch.float32, device="cuda")
    rho = torch.tensor(w.rho, dtype=torch.float32, device="cuda")
    wav = torch.tensor(w.wavelet, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    free = []
    for call in range(2):
        rc = _static_call(lib, w, dm, outs[call], dev=(vp, rho, wav))
        assert rc == 0, lib.lsrtm_last_error().decode()
        free.append(torch.cuda.mem_get_info()[0])
    # (the first call may load kernel code; the second may not take any memory)
    assert free[1] == free[0], ("lsrtm_born_static changed the free device memory", free)
    for call in range(2):
        err = _rel(outs[call], ref)
        assert err < TOL, (call, err)
    # the second call reuses the same static workspace and reproduces the first
    assert _rel(outs[1], outs[0]) < TOL
    # a different problem in between leaves no trace in a later call
    w2 = li.small_case(nz=30, nx=40, nt=150, order=4, npml=6, nshot=2, seed=92)
    d2 = torch.empty((w2.geom.nrec_total, w2.nt), dtype=torch.float32, device="cuda")
    dm2 = torch.tensor(w2.dm, dtype=torch.float32, device="cuda")
    assert _static_call(lib, w2, dm2, d2) == 0
    ref2 = Lsrtm.from_workload(w2).born(dm2)
    assert _rel(d2, ref2) < TOL
    d3 = torch.empty_like(ref)
    assert _static_call(lib, w, dm, d3) == 0
    assert _rel(d3, ref) < TOL


def test_static_born_rejects_oversized_problems():
    from paper_2508_10405_gb300 import load_library
    lib = load_library()
    w = li.small_case(nz=700, nx=700, nt=4, order=8, npml=20, nshot=1, seed=93, hetero=False)
    dm = torch.zeros((2, w.nz, w.nx), dtype=torch.float32, device="cuda")
    d = torch.empty((w.geom.nrec_total, w.nt), dtype=torch.float32, device="cuda")
    rc = _static_call(lib, w, dm, d)
    assert rc == 4   # LSRTM_ERR_OOM
    msg = lib.lsrtm_last_error().decode()
    assert "static" in msg and "bytes" in msg
