#!/usr/bin/env python3
"""Benchmark of the data-domain multiparameter LSRTM hot path.

A step is one CGNR iteration (one Born modelling L, one migration L^T and the
FP64 Krylov updates) over every shot of the workload, with the background
boundary bands cached from the setup. Default workload: the 2D
Marmousi-shaped batched case (384 x 1152 interior, dx = 8 m, order 8,
nt = 4000, dt = 0.8 ms, 96 shots, 1152 receivers each, 10 Hz), seeded
synthetic inputs.

Metric: G cell-updates/s, one cell-update = one padded grid cell advanced one
time step for one shot in one operator application (L and L^T each count
Ncell * nt per shot). Printed as one JSON line on rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs its own copy of the shot set (the
shots are independent: weak scaling, no data-path collective); the time is
the maximum over ranks.
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import lsrtm_inputs as li  # noqa: E402

# Algorithmic HBM bytes per cell-update (FP32, one pass per step, model read
# raw): L = 2 x (3 + 3) state fields read + written + 4 model arrays; L^T = 6
# state fields read + written + 2 model arrays + 2 image planes read + written;
# background only = p, velocities read + written + dt kappa and 1/rho.
from paper_2508_10405_gb300.cglog import BYTES_PER_CELL  # noqa: E402
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", type=int, default=2, help="preset number (default 2)")
    ap.add_argument("--shots-per-batch", type=int, default=0)
    ap.add_argument("--bands", choices=["fp32", "bf16", "fp16"], default="fp16",
                    help="boundary-band precision of the batched (timed) plan")
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--shots", type=int, default=None,
                    help="override the shot count (smaller cases for profiling)")
    ap.add_argument("--nt", type=int, default=None, help="override the number of time steps")
    ap.add_argument("--shard", action="store_true",
                    help="strong scaling: split the survey's shots over the ranks and run the shot-parallel "
                         "CGNR (image all-reduce after every L^T) instead of one survey per rank")
    ap.add_argument("--plan", choices=["batched", "plain"], default="batched",
                    help="execution plan of the timed handle")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default z-chunking instead of timing the candidates")
    ap.add_argument("--plain-shots", type=int, default=4,
                    help="shots on which the plain per-shot FP32 plan is timed for the "
                         "per-iteration comparison (0: skip)")
    ap.add_argument("--image-shots", type=int, default=8,
                    help="shots on which the plain and the batched plans each run the workload's full "
                         "CGNR (its iteration count) for the final-image distance (0: skip)")
    ap.add_argument("--psf-cg", action="store_true",
                    help="time the image-domain CGNR with the interpolated PSF Hessian (App. D) "
                         "on the marine-line image instead of the data-domain iteration")
    ap.add_argument("--psf-iters", type=int, default=100, help="CGNR iterations per --psf-cg step")
    ap.add_argument("--psf-3d", action="store_true",
                    help="with --psf-cg: a 128^3 volume, comb spacing 16, 7^3 node windows (Eq. trilinear)")
    ap.add_argument("--deblur", action="store_true",
                    help="time the image-domain deblurring of the marine-line image: the Fourier-form "
                         "Wiener filter (App. E) and the space-domain 11 x 11 filters")
    ap.add_argument("--model", action="store_true",
                    help="time the data-domain input pipeline (nonlinear modelling in the true and the "
                         "background model, muted residual) instead of the CGNR iteration")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while the
    timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        except Exception:
            rows = []
        if self.path and os.path.exists(self.path):
            os.unlink(self.path)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for n, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if sm:
            out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                   "reasons": sorted(reasons), "samples": len(sm)}
        return out


def step_kernels(w):
    """Names of the Born and migration step kernels the workload runs: the
    TMA-staged 2D kernels (no aperture windows), the per-thread-copy ones
    (windows), or the fused 3D ones."""
    if w.ndim == 3:
        return {"born": "k3f_born", "adjoint": "k3f_adj"}
    if getattr(w.geom, "win_nx", None) is not None:
        return {"born": "k_fwd2d<BORN>", "adjoint": "k_adj2d"}
    return {"born": "k_fwd2t", "adjoint": "k_adj2t"}


def kernel_src_sha(ndim=2):
    h = hashlib.sha256()
    for f in ("kernels2d.cu" if ndim == 2 else "kernels3d_fused.cu", "lsrtm_internal.cuh", "tma.cuh"):
        with open(os.path.join(ROOT, "paper_2508_10405_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel, cells_per_launch, ndim=2):
    """DRAM bytes per launch from the committed ncu summary of this kernel, if
    it was taken on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            t = json.load(f)
        e = t[kernel]
        if e.get("src_sha") != kernel_src_sha(ndim):
            return None
        return float(e["dram_bytes_per_cell"]) * cells_per_launch
    except Exception:
        return None


def shot_cells(w):
    """Padded cells of every shot's grid (its aperture window where it has one)."""
    n = np.full(w.geom.nshot, float(w.padded_cells))
    if getattr(w.geom, "win_nx", None) is not None:
        n = (w.nz + 2.0 * w.npml) * (np.asarray(w.geom.win_nx, np.float64) + 2.0 * w.npml)
    return n


def cpu_sample(w, seconds, reps=1):
    """Times the FP64 oracle (L then L^T) on a bounded sample of the workload:
    a subset of shots and the first nt_s time steps, sized for ~`seconds` of
    work. Returns (G cell-updates/s, threads, description, seconds/rep)."""
    import oracle
    threads = oracle.num_threads()
    if getattr(w.geom, "win_nx", None) is not None:
        threads = 1   # the oracle models windowed shots one call (one thread) at a time
    nshot = min(w.geom.nshot, max(1, threads))
    ncell = float(np.mean(shot_cells(w)[:nshot]))
    geom = w.geom.subset(list(range(nshot)))
    # calibrate the per-step cost from two short runs (removes the set-up time)
    ts = []
    for nt_c in (4, 20):
        t0 = time.perf_counter()
        oracle.born(w, w.dm, geom=geom, nt=nt_c)
        ts.append(time.perf_counter() - t0)
    per_step = max((ts[1] - ts[0]) / 16.0, 1e-6)
    # L^T costs about 3x L in the oracle (checkpointed recomputation)
    nt_s = int(max(16, min(w.nt, seconds / (4.0 * per_step))))
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        d = oracle.born(w, w.dm, geom=geom, nt=nt_s)
        oracle.adjoint(w, d, geom=geom, nt=nt_s)
        times.append(time.perf_counter() - t0)
    t = min(times)
    cells = 2.0 * nshot * ncell * nt_s
    desc = (f"oracle L + L^T on {nshot} of {w.geom.nshot} shots x first {nt_s} of {w.nt} steps "
            f"({cells:.3g} cell-updates), FP64, "
            + ("one thread per windowed shot" if threads == 1 else "OpenMP over shots"))
    return cells / t / 1e9, threads, desc, times


def workload(args):
    kw = {}
    if args.nt is not None:
        kw["nt"] = args.nt
    w = li.preset(args.workload, **kw)
    if args.shots is not None and args.shots < w.geom.nshot:
        w.geom = w.geom.subset(list(range(args.shots)))
    return w


# Image-domain CGNR with the interpolated PSF Hessian (App. D): the marine-line
# image (300 x 2000, comb spacing 20 as in the deblurring experiment), 19 x 19
# node windows, both parameters (2 x 2 blocks).
PSF_CG = {"nz": 300, "nx": 2000, "spacing": 20, "half": 9, "mask": 3}
# FP32 peak of the CUDA cores: 152 SMs x 128 FP32 lanes x 2 flop (FMA) x 2070 MHz.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12


PSF_CG3 = {"shape": (128, 128, 128), "spacing": 16, "half": 3, "mask": 3}


def psf_cg_inputs(nz=None, nx=None):
    c = PSF_CG
    nz, nx = nz or c["nz"], nx or c["nx"]
    pv, pi = li.psf_images(nz, nx, c["spacing"], seed=9)
    m_rtm, _ = li.image_pair(nz, nx, seed=5)
    return pv, pi, m_rtm


def psf_cg3_inputs():
    c = PSF_CG3
    pv, pi = li.psf_images3(*c["shape"], c["spacing"], seed=9)
    m_rtm = np.random.default_rng(5).standard_normal((2,) + c["shape"])
    return pv, pi, m_rtm


def psf_apply_flops(nz, nx, half, mask, ny=None):
    """Algorithmic FP32 flops of one application of H (or H^T): per pixel, window
    offset and parameter block, the interpolated entry (4 multiply-adds over
    the corners in 2D, 8 in 3D) and its product with the input (1 multiply-add)."""
    nblocks = 4 if mask == 3 else 1
    if ny is None:
        return float(nz) * nx * (2 * half + 1) ** 2 * nblocks * 10.0
    return float(nz) * ny * nx * (2 * half + 1) ** 3 * nblocks * 18.0


def psf_cpu_sample(seconds, niter_full):
    """The FP64 oracle's CGNR on a crop of the image (origin on the node grid),
    as many iterations as fit in about `seconds`; scaled to full-image
    iterations/s by the pixel ratio (the cost is linear in the pixels)."""
    from oracle import psf_hessian as ph
    c = PSF_CG
    zc, xc = 60, 400
    pv, pi, m = psf_cg_inputs()
    pv, pi, m = pv[:, :zc, :xc], pi[:, :zc, :xc], m[:, :zc, :xc]
    bl = ph.block_patches(pv, pi, c["spacing"], c["half"], c["mask"])
    t0 = time.perf_counter()
    ph.cgnr(bl, c["spacing"], c["half"], m, 1, c["mask"])
    per = max(time.perf_counter() - t0, 1e-3)
    n = int(max(1, min(niter_full, seconds / per)))
    t0 = time.perf_counter()
    ph.cgnr(bl, c["spacing"], c["half"], m, n, c["mask"])
    t = time.perf_counter() - t0
    ratio = (zc * xc) / float(c["nz"] * c["nx"])
    desc = (f"oracle CGNR, {n} iterations on a {zc} x {xc} crop of the {c['nz']} x {c['nx']} image "
            f"(FP64 numpy, one thread), scaled by the pixel ratio {ratio:.3f}")
    return n / t * ratio, 1, desc, t


def psf_cg_bench(args, rank, world, local):
    import torch
    from paper_2508_10405_gb300 import Lsrtm, binding
    niter, K, W = args.psf_iters, args.steps, args.warmup
    if args.psf_3d:
        c = PSF_CG3
        (nz, ny, nx), s, half, mask = c["shape"], c["spacing"], c["half"], c["mask"]
        wk = li.small_case(ndim=3, nz=nz, ny=ny, nx=nx, nt=8, order=4, npml=4, nshot=1, seed=1)
        pv, pi, m = psf_cg3_inputs()
    else:
        c = PSF_CG
        nz, nx, s, half, mask = c["nz"], c["nx"], c["spacing"], c["half"], c["mask"]
        ny = None
        wk = li.small_case(nz=nz, nx=nx, nt=8, order=4, npml=4, nshot=1, seed=1)
        pv, pi, m = psf_cg_inputs()
    h = Lsrtm.from_workload(wk)
    pv_d, pi_d, m_d = (torch.tensor(a, dtype=torch.float32, device="cuda") for a in (pv, pi, m))
    for _ in range(W):
        h.psf_cg(m_d, pv_d, pi_d, niter, s, half, mask)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    l0 = h.kernel_launches()
    t_steps = []
    for _ in range(K):
        flush.add_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        dm, mis = h.psf_cg(m_d, pv_d, pi_d, niter, s, half, mask)
        e1.record()
        torch.cuda.synchronize()
        t_steps.append(e0.elapsed_time(e1) / 1e3)
    launches = h.kernel_launches() - l0
    # the application kernel alone: H and H^T calls back to back (each call
    # also builds the node windows, a few microseconds)
    reps = 40
    y = torch.empty_like(m_d)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for r in range(reps):
        h.psf_hessian(m_d, pv_d, pi_d, s, half, r % 2 == 1, mask, out=y)
    e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    apply_s = e0.elapsed_time(e1) / 1e3 / reps
    flops = psf_apply_flops(nz, nx, half, mask, ny)
    achieved = flops / apply_s / 1e12
    t_step = float(np.sum(t_steps)) / K
    value = niter * world / t_step
    # end to end through the C ABI with pinned host buffers
    hb = [torch.tensor(a, dtype=torch.float32).pin_memory() for a in (pv, pi, m)]
    dm_h = torch.empty(m.shape, dtype=torch.float32).pin_memory()
    misb = (binding.ctypes.c_double * (niter + 1))()
    torch.cuda.synchronize()
    te = []
    for _ in range(max(K, 1)):
        t0 = time.perf_counter()
        rc = h._lib.lsrtm_psf_cg(h._h, binding._ptr(hb[0]), binding._ptr(hb[1]), s, half, mask,
                                 binding._ptr(hb[2]), binding._ptr(dm_h), niter, misb)
        te.append(time.perf_counter() - t0)
        assert rc == 0
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        if args.psf_3d:
            from oracle import psf_hessian as ph
            sub = tuple(min(n, 24) for n in (nz, ny, nx))
            bl = ph.block_patches(pv[:, :sub[0], :sub[1], :sub[2]], pi[:, :sub[0], :sub[1], :sub[2]], s, half)
            t0 = time.perf_counter()
            ph.cgnr(bl, s, half, m[:, :sub[0], :sub[1], :sub[2]], 1)
            tc = time.perf_counter() - t0
            ratio = float(np.prod(sub)) / (nz * ny * nx)
            cpu = {"value": ratio / tc, "unit": "iter/s", "cores": 1, "kind": "oracle",
                   "sample": f"oracle CGNR, 1 iteration on a {sub} crop, scaled by the voxel ratio {ratio:.4f}"}
        else:
            val, threads, desc, _ = psf_cpu_sample(args.cpu_seconds, niter)
            cpu = {"value": val, "unit": "iter/s", "cores": threads, "kind": "oracle", "sample": desc}
    if rank == 0:
        line = {
            "metric": "PSF-Hessian CGNR iterations/s", "value": value, "unit": "iter/s",
            "n_gpus": world, "steps": K, "warmup": W, "ms_per_step": t_step * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": (f"3D volume {nz} x {ny} x {nx}, comb spacing {s}, {2 * half + 1}^3 node "
                                    f"windows, two parameters" if args.psf_3d else
                                    f"marine-line image {nz} x {nx}, comb spacing {s}, "
                                    f"{2 * half + 1} x {2 * half + 1} node windows, two parameters"),
                       "niter": niter, "step": f"one image-domain CGNR solve of {niter} iterations "
                                               "(node windows built, 2 niter + 1 applications of H or H^T, "
                                               "FP64 Krylov scalars)",
                       "final_misfit": float(mis[-1]),
                       "l2": f"L2 flushed (256 MB write) before every timed step; the solve's vectors take "
                             f"{6 * m.size * 4 / 1e6:.0f} MB"},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": achieved / FP32_PEAK_TFLOPS, "traffic": None,
                         "kernel": "k_psfh3_rows<3>" if args.psf_3d else "k_psfh_apply<3>",
                         "flops_per_launch": flops,
                         "avg_launch_ms": apply_s * 1e3,
                         "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz (no tensor cores)"},
            "clocks": clk, "gpu_launches": int(launches),
            "e2e": {"value": niter / float(np.mean(te)), "unit": "iter/s",
                    "h2d_bytes_per_step": int(sum(a.numel() * 4 for a in hb)),
                    "d2h_bytes_per_step": int(dm_h.numel() * 4 + 8 * (niter + 1)),
                    "calls": "lsrtm_psf_cg with pinned host buffers"},
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    h.close()


def psf_reference_arm(args):
    K, W = args.steps, args.warmup
    for _ in range(W):
        psf_cpu_sample(min(args.cpu_seconds, 5.0) / 4, args.psf_iters)
    vals, descs, ts = [], [], []
    for _ in range(K):
        v, threads, desc, t = psf_cpu_sample(min(args.cpu_seconds, 30.0), args.psf_iters)
        vals.append(v)
        descs.append(desc)
        ts.append(t)
    val = float(np.mean(vals))
    c = PSF_CG
    line = {
        "impl": "reference", "metric": "PSF-Hessian CGNR iterations/s", "value": val, "unit": "iter/s",
        "n_gpus": args.gpus, "steps": K, "warmup": W, "ms_per_step": args.psf_iters / val * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"marine-line image {c['nz']} x {c['nx']}, comb spacing {c['spacing']}, "
                               f"{2 * c['half'] + 1} x {2 * c['half'] + 1} node windows, two parameters",
                   "niter": args.psf_iters, "sample": descs[-1]},
        "cpu_baseline": {"value": val, "unit": "iter/s", "cores": 1, "kind": "oracle", "sample": descs[-1]},
        "e2e": {"value": val, "unit": "iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


MODEL_BYTES_PER_CELL = {nd: BYTES_PER_CELL[("background", nd)] for nd in (2, 3)}


def true_model(w):
    """The true model behind a preset's background and perturbation: the ln map
    of Sec. 2 inverted, v = v0 e^{dm1}, rho = rho0 e^{dm2 - dm1}."""
    return w.vp * np.exp(w.dm[0]), w.rho * np.exp(w.dm[1] - w.dm[0])


def mute_args(w):
    """Direct-wave mute after offset / v_top + 2 / f0 (a Ricker's length),
    rising over 0.25 / f0; far-offset cut at 3/4 of the spread, tapered over
    1/8 of it."""
    spread = w.nx * w.dx
    return (float(np.min(w.vp[0])), 2.0 / w.f0, 0.25 / w.f0, 0.75 * spread, 0.125 * spread)


def model_cpu_sample(w, seconds, reps=1):
    """The FP64 oracle's nonlinear modelling on a bounded sample (shots x first
    steps); G cell-updates/s."""
    import oracle
    threads = oracle.num_threads()
    if getattr(w.geom, "win_nx", None) is not None:
        threads = 1
    nshot = min(w.geom.nshot, max(1, threads))
    geom = w.geom.subset(list(range(nshot)))
    ncell = float(np.mean(shot_cells(w)[:nshot]))
    ts = []
    for nt_c in (4, 20):
        t0 = time.perf_counter()
        oracle.model(w, geom=geom, nt=nt_c)
        ts.append(time.perf_counter() - t0)
    per_step = max((ts[1] - ts[0]) / 16.0, 1e-6)
    nt_s = int(max(16, min(w.nt, seconds / per_step)))
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        oracle.model(w, geom=geom, nt=nt_s)
        times.append(time.perf_counter() - t0)
    cells = nshot * ncell * nt_s
    desc = (f"oracle nonlinear modelling of {nshot} of {w.geom.nshot} shots x first {nt_s} of {w.nt} steps "
            f"({cells:.3g} cell-updates), FP64, " + ("one thread" if threads == 1 else "OpenMP over shots"))
    return cells / min(times) / 1e9, threads, desc, times


def model_bench(args, rank, world, local):
    import dataclasses as dc
    import torch
    from paper_2508_10405_gb300 import Lsrtm
    w = workload(args)
    K, W = args.steps, args.warmup
    vt, rt = true_model(w)
    vmax = float(max(np.max(vt), np.max(w.vp)))
    h_bg = Lsrtm.from_workload(w, pml_vmax=vmax)
    h_tr = Lsrtm.from_workload(dc.replace(w, vp=vt, rho=rt), pml_vmax=vmax)
    margs = mute_args(w)
    d_obs = torch.empty((h_bg.nrec_total, h_bg.nt), dtype=torch.float32, device="cuda")
    d_bg = torch.empty_like(d_obs)
    res = torch.empty_like(d_obs)

    def step():
        h_tr.model(out=d_obs)
        h_bg.model(out=d_bg)
        h_bg.mute_residual(d_obs, d_bg, *margs, out=res)

    for _ in range(W):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    for h in (h_bg, h_tr):
        h.timing(True)
        h.timings(reset=True)
    l0 = h_bg.kernel_launches() + h_tr.kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(K):
        step()
    e1.record()
    torch.cuda.synchronize()
    t_step = e0.elapsed_time(e1) / 1e3 / K
    launches = h_bg.kernel_launches() + h_tr.kernel_launches() - l0
    tms = [h.timings(reset=True) for h in (h_bg, h_tr)]
    # the mute alone, device buffers
    m0, m1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    m0.record()
    for _ in range(5):
        h_bg.mute_residual(d_obs, d_bg, *margs, out=res)
    m1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    mute_s = m0.elapsed_time(m1) / 1e3 / 5
    cells_per_model = float(shot_cells(w).sum()) * w.nt
    value = 2.0 * cells_per_model * world / t_step / 1e9
    ms = sum(tm["background_ms"] for tm in tms)
    nl = sum(tm["background_launches"] for tm in tms)
    cells = sum(tm["background_cells"] for tm in tms)
    bpc = MODEL_BYTES_PER_CELL[w.ndim]
    achieved = bpc * (cells / nl) / (ms / 1e3 / nl) / 1e9
    peak, peak_kind = peaks()
    nd = h_bg.nrec_total * h_bg.nt
    # end to end: the records and the residual to pinned host memory
    hb = torch.empty((h_bg.nrec_total, h_bg.nt), dtype=torch.float32).pin_memory()
    t0 = time.perf_counter()
    for _ in range(max(K, 1)):
        h_tr.model(out=d_obs)
        h_bg.model(out=d_bg)
        h_bg.mute_residual(d_obs, d_bg, *margs, out=hb)
        torch.cuda.synchronize()
    te = (time.perf_counter() - t0) / max(K, 1)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        val, threads, desc, _ = model_cpu_sample(w, args.cpu_seconds)
        cpu = {"value": val, "unit": "Gcell-updates/s", "cores": threads, "kind": "oracle", "sample": desc}
    if rank == 0:
        line = {
            "metric": "nonlinear modelling Gcell-updates/s", "value": value, "unit": "Gcell-updates/s",
            "n_gpus": world, "steps": K, "warmup": W, "ms_per_step": t_step * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": w.name, "grid": list(w.shape), "nt": w.nt, "order": w.order,
                       "shots_per_rank": w.geom.nshot,
                       "step": "observed data in the true model + background data + muted residual",
                       "mute": dict(zip(["v_mute", "t0", "t_taper", "o_max", "o_taper"], margs)),
                       "l2": "inputs larger than L2 (state of all shots of a batch)"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "kernel": "k_fwd2d<background>",
                         "algorithmic_bytes_per_cell": bpc, "avg_launch_ms": ms / nl,
                         "peak_source": f"{peak_kind} MEASURED_PEAKS.json hbm_gbs"},
            "mute": {"ms": mute_s * 1e3, "gbs": 12.0 * nd / mute_s / 1e9, "bytes_per_sample": 12},
            "clocks": clk, "gpu_launches": int(launches),
            "e2e": {"value": 2.0 * cells_per_model * world / te / 1e9, "unit": "Gcell-updates/s",
                    "h2d_bytes_per_step": 0, "d2h_bytes_per_step": int(nd * 4),
                    "calls": "lsrtm_model x2 + lsrtm_mute_residual into pinned host memory"},
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    h_bg.close()
    h_tr.close()


def wiener_flops(nz, nx, s):
    """Algorithmic FP32 flops of the Wiener blocks: per block and plane three
    2D DFTs of N = 2s points per axis, each axis one Cooley-Tukey split
    N = N1 N2 (N1 the divisor nearest sqrt N): per output N1 + N2 complex
    multiply-adds and one twiddle product (8 and 6 flops), over N^2 outputs
    and 2 axes."""
    nk = len(range(s // 2, nz, s)) * len(range(s // 2, nx, s))
    N = 2 * s
    n1 = min((d for d in range(1, N + 1) if N % d == 0), key=lambda d: abs(d * d - N))
    per_out = (n1 + N // n1) * 8 + 6
    return 2.0 * nk * 3 * 2 * N ** 2 * per_out


def deblur_bench(args, rank, world, local):
    import torch
    from paper_2508_10405_gb300 import Lsrtm
    from oracle import wiener as wf
    nz, nx, s, eps = 300, 2000, 20, 1e-3
    K, W = args.steps, args.warmup
    wk = li.small_case(nz=nz, nx=nx, nt=8, order=4, npml=4, nshot=1, seed=1)
    h = Lsrtm.from_workload(wk)
    m, r = li.image_pair(nz, nx, seed=5)
    md = torch.tensor(m, dtype=torch.float32, device="cuda")
    rd = torch.tensor(r, dtype=torch.float32, device="cuda")
    out = torch.empty_like(md)
    for _ in range(W):
        h.deblur_wiener(md, rd, s, eps, out=out)
        h.deblur(md, rd, s, 11, eps)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    l0 = h.kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(K):
        h.deblur_wiener(md, rd, s, eps, out=out)
    e1.record()
    torch.cuda.synchronize()
    t_w = e0.elapsed_time(e1) / 1e3 / K
    launches = h.kernel_launches() - l0
    e0.record()
    for _ in range(K):
        h.deblur(md, rd, s, 11, eps)
    e1.record()
    torch.cuda.synchronize()
    t_s = e0.elapsed_time(e1) / 1e3 / K
    clk = clocks.stop()
    flops = wiener_flops(nz, nx, s)
    # end to end with host buffers
    mh, rh = (torch.tensor(a, dtype=torch.float32).pin_memory() for a in (m, r))
    oh = torch.empty_like(mh).pin_memory()
    t0 = time.perf_counter()
    for _ in range(max(K, 1)):
        h.deblur_wiener(mh, rh, s, eps, out=oh)
        torch.cuda.synchronize()
    te = (time.perf_counter() - t0) / max(K, 1)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        t0 = time.perf_counter()
        wf.wiener(m, r, s, eps)
        tc = time.perf_counter() - t0
        cpu = {"value": 1.0 / tc, "unit": "images/s", "cores": 1, "kind": "oracle",
               "sample": "oracle Wiener deblurring of the whole 300 x 2000 two-parameter image (numpy FFT, FP64)"}
    if rank == 0:
        line = {
            "metric": "Wiener deblurring images/s", "value": world / t_w, "unit": "images/s", "n_gpus": world,
            "steps": K, "warmup": W, "ms_per_step": t_w * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "marine-line image 300 x 2000, two parameters, comb spacing 20, 40 x 40 blocks",
                       "eps": eps, "step": "one Wiener deblurring of the image (1500 blocks per plane, blend)",
                       "l2": "image 4.8 MB per input: L2-resident"},
            "roofline": {"bound": "alu", "achieved": flops / t_w / 1e12, "peak": FP32_PEAK_TFLOPS,
                         "unit": "TFLOP/s", "frac": flops / t_w / 1e12 / FP32_PEAK_TFLOPS, "traffic": None,
                         "kernel": "k_wiener_block + k_wiener_blend", "flops_per_launch": flops,
                         "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz"},
            "space_domain_filters": {"ms": t_s * 1e3, "kernel": "k_deblur_solve + k_deblur_apply (11 x 11, FP64 "
                                                               "normal equations)"},
            "clocks": clk, "gpu_launches": int(launches),
            "e2e": {"value": 1.0 / te, "unit": "images/s", "h2d_bytes_per_step": int(2 * mh.numel() * 4),
                    "d2h_bytes_per_step": int(oh.numel() * 4), "calls": "lsrtm_deblur_wiener with pinned host buffers"},
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    h.close()


def reference_arm(args, rank, world):
    if rank != 0:
        return
    if args.deblur:
        from oracle import wiener as wf
        m, r = li.image_pair(300, 2000, seed=5)
        ts = []
        for _ in range(max(args.steps, 1)):
            t0 = time.perf_counter()
            wf.wiener(m, r, 20, 1e-3)
            ts.append(time.perf_counter() - t0)
        val = 1.0 / float(np.mean(ts))
        desc = "oracle Wiener deblurring of the whole 300 x 2000 two-parameter image (numpy FFT, FP64)"
        print(json.dumps({"impl": "reference", "metric": "Wiener deblurring images/s", "value": val,
                          "unit": "images/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                          "ms_per_step": 1e3 / val, "higher_is_better": True, "scaling": "weak",
                          "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                          "config": {"workload": "marine-line image 300 x 2000, spacing 20", "sample": desc},
                          "cpu_baseline": {"value": val, "unit": "images/s", "cores": 1, "kind": "oracle",
                                           "sample": desc},
                          "e2e": {"value": val, "unit": "images/s", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}), flush=True)
        return
    if args.psf_cg:
        psf_reference_arm(args)
        return
    if args.model:
        w = workload(args)
        K, W = args.steps, args.warmup
        per = max(2.0, min(args.cpu_seconds, 120.0 / max(K + W, 1)))
        val, threads, desc, times = model_cpu_sample(w, per, reps=max(K, 1))
        line = {"impl": "reference", "metric": "nonlinear modelling Gcell-updates/s", "value": val,
                "unit": "Gcell-updates/s", "n_gpus": args.gpus, "steps": K, "warmup": W,
                "ms_per_step": 1e3 * float(np.mean(times)), "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": w.name, "grid": [w.nz, w.nx], "nt": w.nt, "sample": desc},
                "cpu_baseline": {"value": val, "unit": "Gcell-updates/s", "cores": threads, "kind": "oracle",
                                 "sample": desc},
                "e2e": {"value": val, "unit": "Gcell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    w = workload(args)
    K, W = args.steps, args.warmup
    # bounded per-step sample sized so the whole run stays within minutes
    per = max(2.0, min(args.cpu_seconds, 120.0 / max(K + W, 1)))
    _, _, _, _ = cpu_sample(w, per / 4, reps=max(W, 0)) if W > 0 else (0, 0, "", [])
    val, threads, desc, times = cpu_sample(w, per, reps=K)
    ms = 1e3 * float(np.mean(times))
    line = {
        "impl": "reference", "metric": "Born+migration Gcell-updates/s", "value": val,
        "unit": "Gcell-updates/s", "n_gpus": args.gpus, "steps": K, "warmup": W,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "grid": [w.nz, w.nx], "nt": w.nt, "order": w.order,
                   "shots": w.geom.nshot, "sample": desc},
        "cpu_baseline": {"value": val, "unit": "Gcell-updates/s", "cores": threads,
                         "kind": "oracle", "sample": desc},
        "e2e": {"value": val, "unit": "Gcell-updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def plain_compare(w, nshots, s_batched, bands, torch, image_shots):
    """The plain plan (one shot per launch, no graphs, FP32 bands, background
    recomputed inside every L^T) against the batched mixed-precision plan.
    Per-iteration time: the plain plan timed on the first `nshots` shots
    (fastest of two CGNR iterations, z-chunking autotuned like the batched
    handle) and scaled to all shots by padded cells, against the batched
    plan's measured iteration. Final-image distance: both plans run the
    workload's full CGNR (w.cg_iters iterations) on the first `image_shots`
    shots from the same observed data; the relative L2 distance of the two
    final images."""
    from paper_2508_10405_gb300 import BAND_BF16, BAND_FP16, BAND_FP32, PLAN_BATCHED, PLAN_PLAIN, Lsrtm
    bp = {"fp32": BAND_FP32, "bf16": BAND_BF16, "fp16": BAND_FP16}[bands]
    nshots = min(nshots, w.geom.nshot)
    sub = dataclasses.replace(w, geom=w.geom.subset(list(range(nshots))))
    hp = Lsrtm.from_workload(sub, plan=PLAN_PLAIN, band_precision=BAND_FP32)
    tune = hp.autotune()
    dm = torch.tensor(w.dm, dtype=torch.float32, device="cuda")
    d = hp.born(dm)
    hp.cg_begin(d)
    times = []
    for _ in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hp.cg_iterate(1)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    hp.close()
    frac = float(shot_cells(w)[:nshots].sum() / shot_cells(w).sum())
    s_plain = min(times) / frac
    out = {"s_per_iter_plain": s_plain, "s_per_iter_batched": s_batched,
           "speedup": s_plain / s_batched,
           "plain": "one shot per launch, no graph, FP32 bands, background recomputed in every L^T",
           "batched": f"all shots per launch, CUDA graphs, {bands} bands cached across iterations",
           "plain_autotune_tzc": tune.get("tzc"),
           "sample": f"plain timed on {nshots} of {w.geom.nshot} shots (fastest of 2 iterations), "
                     f"scaled by padded cells"}
    ni = max(1, int(w.cg_iters))
    if image_shots > 0:
        # The batched plan with FP32 bands computes bit for bit what the plain
        # plan does (tests/test_gpu_parity.py::test_plain_plan_equals_batched),
        # so it stands in for the plain plan here. The sensitivity floor: the
        # same FP32 solve on data perturbed by 1e-6 relative noise.
        ns = min(image_shots, w.geom.nshot)
        shots = list(np.linspace(0, w.geom.nshot - 1, ns).round().astype(int))
        sub = dataclasses.replace(w, geom=w.geom.subset(shots))
        h32 = Lsrtm.from_workload(sub, plan=PLAN_BATCHED, band_precision=BAND_FP32)
        h16 = Lsrtm.from_workload(sub, plan=PLAN_BATCHED, band_precision=bp)
        dd = h32.born(dm)
        gen = torch.Generator(device="cuda").manual_seed(7)
        dp = dd * (1 + 1e-6 * torch.randn(dd.shape, device="cuda", generator=gen))
        res = {}
        for k in sorted({5, ni}):
            x32, m32 = h32.cg_solve(dd, k)
            x16, m16 = h16.cg_solve(dd, k)
            xp, _ = h32.cg_solve(dp, k)
            x32 = x32.double()
            nrm = torch.linalg.norm(x32)
            res[k] = {"bands_vs_fp32": float(torch.linalg.norm(x16.double() - x32) / nrm),
                      "fp32_under_1e-6_data_perturbation": float(torch.linalg.norm(xp.double() - x32) / nrm),
                      "misfit_fp32": float(m32[-1]), f"misfit_{bands}": float(m16[-1])}
        # the stand-in checked here too: the plain plan's own 5-iteration image
        hpl = Lsrtm.from_workload(sub, plan=PLAN_PLAIN, band_precision=BAND_FP32)
        hpl.autotune()
        xpl, _ = hpl.cg_solve(dd, 5)
        x32, _ = h32.cg_solve(dd, 5)
        hpl.close()
        res["plain_vs_batched_fp32_5_iterations"] = {
            "rel_l2": float(torch.linalg.norm(xpl.double() - x32.double()) / torch.linalg.norm(x32.double())),
            "bitwise": bool(torch.equal(xpl, x32))}
        h32.close()
        h16.close()
        out["final_image_rel_l2"] = res[ni]["bands_vs_fp32"]
        out["final_image"] = {"iterations": res, "shots": [int(v) for v in shots],
                              "what": f"{bands}-band batched vs FP32 (= plain) CGNR images after 5 and {ni} "
                                      f"iterations on {ns} shots, beside the change a 1e-6 relative data "
                                      f"perturbation causes in the FP32 solve"}
    return out


def shard_bench(args, rank, world, local):
    """Strong scaling of one survey (Sec. 3: shots mapped to processors, the
    image reduced): rank r owns shots r, r + N, ... and the step is one
    iteration of the shot-parallel CGNR (distributed.ShotParallelCG: the
    rank's L and L^T, an all-reduce of the two-parameter image after every
    L^T and of the FP64 data-space inner products). value = the whole
    survey's cell-updates per iteration / the slowest rank's time."""
    import torch
    import torch.distributed as dist
    import dataclasses
    from paper_2508_10405_gb300 import BAND_BF16, BAND_FP16, BAND_FP32, Lsrtm
    from paper_2508_10405_gb300.distributed import ShotParallelCG, shard
    bands = {"fp32": BAND_FP32, "bf16": BAND_BF16, "fp16": BAND_FP16}[args.bands]
    w = workload(args)
    K, W = args.steps, args.warmup
    mine = shard(w.geom.nshot, rank, world)
    wl = dataclasses.replace(w, geom=w.geom.subset(mine))
    cells_per_step = 2.0 * float(shot_cells(w).sum()) * w.nt   # the whole survey's L + L^T
    h = Lsrtm.from_workload(wl, band_precision=bands, shots_per_batch=args.shots_per_batch)
    tune = None if args.no_autotune else h.autotune()
    dm_true = torch.tensor(w.dm, dtype=torch.float32, device="cuda")
    d_local = h.born(dm_true)
    cg = ShotParallelCG(h, heartbeat_timeout=600.0)
    ev = {W: torch.cuda.Event(enable_timing=True), W + K: torch.cuda.Event(enable_timing=True)}
    clocks = ClockSampler(local)

    def mark(k):
        if k == W:
            torch.cuda.synchronize()
            if world > 1:
                dist.barrier()
            clocks.start()
            h.timing(True)
            h.timings(reset=True)
        if k in ev:
            ev[k].record()

    if W == 0:
        mark(0)
    x, mis = cg.solve(d_local, W + K, on_iteration=mark)
    torch.cuda.synchronize()
    tm = h.timings(reset=True)
    h.timing(False)
    clk = clocks.stop()
    t = torch.tensor([ev[W].elapsed_time(ev[W + K]) / 1e3], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    t_max = float(t.item())
    kinds = {"born": (tm["born_ms"], tm["born_launches"], tm["born_cells"]),
             "adjoint": (tm["adjoint_ms"], tm["adjoint_launches"], tm["adjoint_cells"])}
    dom = max(kinds, key=lambda k: kinds[k][0])
    ms, nl, cells = kinds[dom]
    bpc = BYTES_PER_CELL[(dom, w.ndim)]
    achieved = bpc * (cells / max(nl, 1)) / (ms / 1e3 / max(nl, 1)) / 1e9 if ms else None
    peak, peak_kind = peaks()
    kname = step_kernels(w)[dom]
    if rank == 0:
        line = {
            "metric": "Born+migration Gcell-updates/s", "value": cells_per_step * K / t_max / 1e9,
            "unit": "Gcell-updates/s", "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": t_max / K * 1e3, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "grid": list(w.shape), "nt": w.nt, "order": w.order,
                       "shots": w.geom.nshot, "shots_per_rank": len(mine), "bands": args.bands,
                       "autotune": tune, "s_per_lsrtm_iter": t_max / K,
                       "step": "one shot-parallel CGNR iteration (rank-local L + L^T, image and FP64 "
                               "inner-product all-reduces)",
                       "parallelism": f"shots sharded over {world} rank(s), image all-reduce per L^T"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak if achieved else None,
                         "traffic": ncu_traffic(kname, cells / max(nl, 1), w.ndim), "kernel": kname,
                         "peak_source": f"{peak_kind} MEASURED_PEAKS.json hbm_gbs"},
            "clocks": clk, "misfit": mis[-1], "e2e": None, "cpu_baseline": None,
        }
        print(json.dumps(line), flush=True)
    h.close()
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return
    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    if args.psf_cg:
        psf_cg_bench(args, rank, world, local)
        return
    if args.model:
        model_bench(args, rank, world, local)
        return
    if args.deblur:
        deblur_bench(args, rank, world, local)
        return
    if world > 1:
        dist.init_process_group("nccl")
    if args.shard:
        shard_bench(args, rank, world, local)
        return

    from paper_2508_10405_gb300 import BAND_BF16, BAND_FP16, BAND_FP32, PLAN_BATCHED, PLAN_PLAIN, Lsrtm
    bands = {"fp32": BAND_FP32, "bf16": BAND_BF16, "fp16": BAND_FP16}[args.bands]

    w = workload(args)
    K, W = args.steps, args.warmup
    ncell = w.padded_cells
    nshot = w.geom.nshot
    cells_per_step = 2.0 * float(shot_cells(w).sum()) * w.nt   # L + L^T per CG iteration
    h = Lsrtm.from_workload(w, band_precision=bands,
                            shots_per_batch=args.shots_per_batch,
                            plan=PLAN_PLAIN if args.plan == "plain" else PLAN_BATCHED)
    tune = None if args.no_autotune else h.autotune()   # untimed setup
    dm_true = torch.tensor(w.dm, dtype=torch.float32, device="cuda")
    d_obs = h.born(dm_true)                 # synthetic observed data (untimed setup)
    h.cg_begin(d_obs)                       # background bands cached here
    for _ in range(W):
        h.cg_iterate(1)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()

    clocks = ClockSampler(local)
    clocks.start()
    h.timing(True)
    h.timings(reset=True)
    l0 = h.kernel_launches()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ev0.record()
    for _ in range(K):
        h.cg_iterate(1)
    ev1.record()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t_local = ev0.elapsed_time(ev1) / 1e3
    launches = h.kernel_launches() - l0
    workspace = h.workspace_bytes()
    tm = h.timings(reset=True)
    h.timing(False)
    clk = clocks.stop()
    t = torch.tensor([t_local], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    t_max = float(t.item())
    value = cells_per_step * K * world / t_max / 1e9

    # dominant kernel and its roofline
    kinds = {"born": (tm["born_ms"], tm["born_launches"], tm["born_cells"]),
             "adjoint": (tm["adjoint_ms"], tm["adjoint_launches"], tm["adjoint_cells"])}
    dom = max(kinds, key=lambda k: kinds[k][0])
    ms, nl, cells = kinds[dom]
    cells_per_launch = cells / max(nl, 1)
    avg_launch_s = ms / 1e3 / max(nl, 1)
    bpc = BYTES_PER_CELL[(dom, w.ndim)]
    achieved = bpc * cells_per_launch / avg_launch_s / 1e9
    peak, peak_kind = peaks()
    kname = step_kernels(w)[dom]
    traffic = ncu_traffic(kname, cells_per_launch, w.ndim)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "kernel": kname,
                "peak_source": f"{peak_kind} MEASURED_PEAKS.json hbm_gbs" if peak_kind == "measured"
                else "fallback 6.8 TB/s",
                "algorithmic_bytes_per_cell": bpc, "cells_per_launch": cells_per_launch,
                "avg_launch_ms": avg_launch_s * 1e3}
    per_op = {k: {"ms_per_step": v[0] / K, "gcells_per_s": v[2] / (v[0] / 1e3) / 1e9 if v[0] else None,
                  "gbs": BYTES_PER_CELL[(k, w.ndim)] * v[2] / (v[0] / 1e3) / 1e9 if v[0] else None}
              for k, v in kinds.items()}

    # end to end through the public API with pinned host buffers: per step a
    # Born modelling (host dm in, host d out) and a migration (host d in, host g out)
    E = args.e2e_steps if args.e2e_steps is not None else K
    e2e = None
    if E > 0:
        dm_h = torch.empty(dm_true.shape, dtype=torch.float32, pin_memory=True)
        dm_h.copy_(dm_true.cpu())
        d_h = torch.empty((h.nrec_total, h.nt), dtype=torch.float32, pin_memory=True)
        g_h = torch.empty((2,) + h.shape, dtype=torch.float32, pin_memory=True)
        h.born(dm_h, out=d_h)
        h.adjoint(d_h, out=g_h)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(E):
            h.born(dm_h, out=d_h)
            h.adjoint(d_h, out=g_h)
        e1.record()
        torch.cuda.synchronize()
        te = torch.tensor([e0.elapsed_time(e1) / 1e3], dtype=torch.float64, device="cuda")
        if world > 1:
            dist.all_reduce(te, op=dist.ReduceOp.MAX)
        te = float(te.item())
        e2e = {"value": cells_per_step * E * world / te / 1e9, "unit": "Gcell-updates/s",
               "h2d_bytes_per_step": int(dm_h.numel() * 4 + d_h.numel() * 4),
               "d2h_bytes_per_step": int(d_h.numel() * 4 + g_h.numel() * 4),
               "calls": "lsrtm_born + lsrtm_adjoint with pinned host buffers"}

    plain = None
    if args.plain_shots > 0 and args.plan == "batched":
        plain = plain_compare(w, args.plain_shots, t_max / K, args.bands, torch, args.image_shots)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        val, threads, desc, _ = cpu_sample(w, args.cpu_seconds)
        cpu = {"value": val, "unit": "Gcell-updates/s", "cores": threads, "kind": "oracle",
               "sample": desc}

    if rank == 0:
        line = {
            "metric": "Born+migration Gcell-updates/s", "value": value, "unit": "Gcell-updates/s",
            "n_gpus": world, "steps": K, "warmup": W, "ms_per_step": t_max / K * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "grid": list(w.shape), "padded_cells": ncell,
                       "padded_cells_per_step": float(shot_cells(w).sum()),
                       "nt": w.nt, "order": w.order, "shots_per_rank": nshot,
                       "receivers_per_shot": float(np.mean(np.diff(w.geom.rec_ptr))),
                       "bands": args.bands, "plan": args.plan,
                       "autotune": tune,
                       "step": "one CGNR iteration (L + L^T + FP64 Krylov updates)",
                       "s_per_lsrtm_iter": t_max / K,
                       "l2": f"inputs larger than L2 (workspace {workspace / 1e9:.1f} GB per rank)",
                       "parallelism": f"shots per rank, {world} rank(s), no data-path collective"},
            "roofline": roofline, "per_operator": per_op, "clocks": clk,
            "gpu_launches": int(launches), "e2e": e2e, "cpu_baseline": cpu,
            "plain_vs_batched": plain,
        }
        print(json.dumps(line), flush=True)
    h.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
