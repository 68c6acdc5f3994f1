"""Seeded synthetic inputs for the LSRTM operator pair.

This module only draws and shapes inputs: velocity and density models, model
perturbations, source wavelets and acquisition geometry, and the synthetic
images of the image-domain steps (a migrated image and its blurred
remigration, the PSF images of spike combs in 2D and 3D). It contains none of
the operator arithmetic (no stencils, no model preparation, no absorbing
boundary, no interpolation or filtering), so both the FP64 oracle and the
CUDA path can take their inputs from it without sharing any of the method.

The five workload presets stand in for the paper's Marmousi 2D, Overthrust 3D
and Viking Graben experiments (Sec. 4 and Sec. 6), none of which is available
here; each preset copies the shape class of its experiment (grid size, order,
shot and receiver layout, frequency) with seeded random structure.

Array conventions (shared by every consumer):
  * interior models are float64 arrays shaped [nz, nx] (2D) or [nz, ny, nx]
    (3D), x fastest;
  * a flat interior index is (iz*ny + iy)*nx + ix (ny = 1 in 2D);
  * a model perturbation is [2, nz, (ny,) nx] with plane 0 = dln Vp and
    plane 1 = dln Ip (the paper's (m1, m2), Sec. 2);
  * geometry: one source node per shot (flat interior index) and receivers in
    CSR form rec_ptr[nshot+1], rec_idx[rec_ptr[-1]];
  * data are [rec_ptr[-1], nt], receiver-major with contiguous time.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Workload", "Geometry", "preset", "PRESETS", "ricker", "gardner_rho",
    "gaussian_blobs", "small_case", "image_pair", "psf_images", "psf_images3",
]


@dataclasses.dataclass
class Geometry:
    src_idx: np.ndarray   # int32 [nshot]
    rec_ptr: np.ndarray   # int32 [nshot+1]
    rec_idx: np.ndarray   # int32 [rec_ptr[-1]]
    win_x0: np.ndarray | None = None  # int32 [nshot] aperture start (interior x) or None
    win_nx: np.ndarray | None = None  # int32 [nshot] aperture width or None

    @property
    def nshot(self) -> int:
        return int(self.src_idx.shape[0])

    @property
    def nrec_total(self) -> int:
        return int(self.rec_ptr[-1])

    def subset(self, shots) -> "Geometry":
        """Geometry restricted to the listed shots (kept in the given order)."""
        shots = np.asarray(shots, dtype=np.int64)
        ptr = [0]
        idx = []
        for s in shots:
            r = self.rec_idx[self.rec_ptr[s]:self.rec_ptr[s + 1]]
            idx.append(r)
            ptr.append(ptr[-1] + r.size)
        return Geometry(
            src_idx=self.src_idx[shots].astype(np.int32),
            rec_ptr=np.asarray(ptr, dtype=np.int32),
            rec_idx=(np.concatenate(idx) if idx else np.zeros(0)).astype(np.int32),
            win_x0=None if self.win_x0 is None else self.win_x0[shots].astype(np.int32),
            win_nx=None if self.win_nx is None else self.win_nx[shots].astype(np.int32),
        )


@dataclasses.dataclass
class Workload:
    name: str
    ndim: int
    nz: int
    ny: int
    nx: int
    dz: float
    dy: float
    dx: float
    dt: float
    nt: int
    order: int
    npml: int
    f0: float
    vp: np.ndarray        # background velocity, interior
    rho: np.ndarray       # background density, interior
    dm: np.ndarray        # [2, ...] reference perturbation (dln Vp, dln Ip)
    wavelet: np.ndarray   # [nt] source time function samples w(n*dt)
    geom: Geometry
    cg_iters: int = 0
    notes: str = ""
    free_surface: bool = False   # free surface on the first interior row

    @property
    def shape(self):
        return (self.nz, self.nx) if self.ndim == 2 else (self.nz, self.ny, self.nx)

    @property
    def nint(self) -> int:
        return self.nz * self.ny * self.nx

    @property
    def padded_cells(self) -> int:
        n = (self.nz + 2 * self.npml) * (self.nx + 2 * self.npml)
        if self.ndim == 3:
            n *= self.ny + 2 * self.npml
        return n


def ricker(nt: int, dt: float, f0: float, delay: float | None = None) -> np.ndarray:
    """Ricker wavelet w(t) = (1 - 2 pi^2 f0^2 tau^2) exp(-pi^2 f0^2 tau^2),
    tau = t - delay, sampled at t = n*dt; delay defaults to 1/f0."""
    t = np.arange(nt, dtype=np.float64) * dt
    tau = t - (1.0 / f0 if delay is None else delay)
    a = (math.pi * f0 * tau) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def gardner_rho(vp: np.ndarray) -> np.ndarray:
    """Gardner's relation rho = 310 * v^0.25 (SI units), as the paper uses for
    the Viking Graben density (Sec. 6)."""
    return 310.0 * np.power(vp, 0.25)


def gaussian_blobs(rng, shape, n, sigma_cells, amp_range, lo, hi):
    """Sum of n isotropic Gaussian blobs with centres drawn U[lo, hi] per axis
    and amplitudes U[amp_range]."""
    grids = np.meshgrid(*[np.arange(s, dtype=np.float64) for s in shape], indexing="ij")
    out = np.zeros(shape)
    centres = rng.uniform(lo, hi, size=(n, len(shape)))
    amps = rng.uniform(amp_range[0], amp_range[1], size=n)
    for c, a in zip(centres, amps):
        r2 = sum((g - ci) ** 2 for g, ci in zip(grids, c))
        out += a * np.exp(-0.5 * r2 / sigma_cells ** 2)
    return out, centres


def _smooth(a: np.ndarray, sigma_cells: float) -> np.ndarray:
    from scipy.ndimage import gaussian_filter
    return gaussian_filter(a, sigma_cells, mode="nearest")


def _flat(ndim, ny, nx, iz, iy, ix):
    return (np.asarray(iz) * ny + np.asarray(iy)) * nx + np.asarray(ix)


def _surface_line_geometry(nz, nx, src_x, rec_x_lists, src_z=1, rec_z=1):
    src = np.asarray([_flat(2, 1, nx, src_z, 0, x) for x in src_x], dtype=np.int32)
    ptr = [0]
    idx = []
    for rx in rec_x_lists:
        rx = np.asarray(rx, dtype=np.int64)
        idx.append(_flat(2, 1, nx, rec_z, 0, rx))
        ptr.append(ptr[-1] + rx.size)
    return Geometry(src, np.asarray(ptr, np.int32), np.concatenate(idx).astype(np.int32))


# --------------------------------------------------------------------------
# Presets. Each builder takes a seed (default = preset number) and optional
# overrides of the grid (used by tests to shrink a workload while keeping its
# structure).
# --------------------------------------------------------------------------

def _cfg1(seed=1, nz=101, nx=101, nt=1000):
    """2D plain Born+migration: linear v(z), Gardner rho, 1 surface shot at the
    centre, 101 receivers at z = 10 m, three Gaussian blobs in both planes."""
    rng = np.random.default_rng(seed)
    dx = 10.0
    z = np.arange(nz, dtype=np.float64)[:, None] * np.ones((1, nx))
    vp = 1500.0 + 1000.0 * z / max(nz - 1, 1)
    rho = gardner_rho(vp)
    sig = 30.0 / dx
    lo, hi = 0.2 * (nz - 1), 0.8 * (nz - 1)
    grids = np.meshgrid(np.arange(nz, dtype=np.float64), np.arange(nx, dtype=np.float64), indexing="ij")
    centres = rng.uniform(lo, hi, size=(3, 2))
    dm = np.zeros((2, nz, nx))
    for p in range(2):
        amps = rng.uniform(-0.05, 0.05, size=3)
        for c, a in zip(centres, amps):
            r2 = (grids[0] - c[0]) ** 2 + (grids[1] - c[1]) ** 2
            dm[p] += a * np.exp(-0.5 * r2 / sig ** 2)
    geom = _surface_line_geometry(nz, nx, [nx // 2], [np.arange(nx)], src_z=0, rec_z=1)
    dt = 1e-3
    return Workload("cfg1_2d_plain", 2, nz, 1, nx, dx, dx, dx, dt, nt, 4, 20, 15.0,
                    vp, rho, dm, ricker(nt, dt, 15.0), geom,
                    notes="linear v(z) 1500-2500 m/s, Gardner rho, 3 Gaussian blobs (sigma 30 m)")


def _layered_faulted(rng, nz, nx, nlayers, vmin, vmax, nfaults, throw_range, undul_amp):
    """Layer-cake velocity with sinusoidal undulation, +-5% jitter per layer and
    normal faults (vertical offsets of the layer index to one side of a dipping
    fault line)."""
    z = np.arange(nz, dtype=np.float64)[:, None]
    x = np.arange(nx, dtype=np.float64)[None, :]
    bounds = np.sort(rng.uniform(0.04 * nz, nz, size=nlayers - 1))
    k1, k2 = rng.uniform(1.0, 4.0, size=2) * 2 * math.pi / nx
    ph = rng.uniform(0, 2 * math.pi, size=2)
    undul = undul_amp * (np.sin(k1 * x + ph[0]) + 0.5 * np.sin(k2 * x + ph[1]))
    zz = z - undul * (z / nz)
    for _ in range(nfaults):
        xf = rng.uniform(0.15 * nx, 0.85 * nx)
        slope = rng.uniform(0.3, 0.8) * rng.choice([-1.0, 1.0])
        throw = rng.uniform(*throw_range)
        side = (x - xf) > slope * z
        zz = np.where(side, zz - throw, zz)
    layer = np.searchsorted(bounds, zz)
    base = np.linspace(vmin, vmax, nlayers)
    jitter = 1.0 + rng.uniform(-0.05, 0.05, size=nlayers)
    vl = np.clip(base * jitter, vmin, vmax)
    vl[0] = vmin
    return vl[np.clip(layer, 0, nlayers - 1)]


def _true_to_background(vt, rhot, sigma_cells):
    v0 = _smooth(vt, sigma_cells)
    r0 = _smooth(rhot, sigma_cells)
    dm = np.stack([np.log(vt) - np.log(v0), np.log(vt * rhot) - np.log(v0 * r0)])
    return v0, r0, dm


def _cfg2(seed=2, nz=384, nx=1152, nt=4000, nshot=96, shot_dx=12, shot_x0=6):
    """2D Marmousi-shaped batched LSRTM: faulted layers 1500-4700 m/s, Gardner
    rho, background = 200 m Gaussian smoothing, dm from the unsmoothed model,
    96 shots every 96 m, receivers at every surface cell."""
    rng = np.random.default_rng(seed)
    dx = 8.0
    vt = _layered_faulted(rng, nz, nx, 25, 1500.0, 4700.0, 3, (3, 8), 0.02 * nz)
    rhot = gardner_rho(vt)
    v0, r0, dm = _true_to_background(vt, rhot, 200.0 / dx)
    xs = [min(shot_x0 + shot_dx * k, nx - 1) for k in range(nshot)]
    geom = _surface_line_geometry(nz, nx, xs, [np.arange(nx)] * nshot, src_z=1, rec_z=1)
    dt = 0.8e-3
    return Workload("cfg2_2d_marmousi_like", 2, nz, 1, nx, dx, dx, dx, dt, nt, 8, 20, 10.0,
                    v0, r0, dm, ricker(nt, dt, 10.0), geom, cg_iters=20,
                    notes="seeded faulted layers (25 layers, 3 faults), 200 m smoothing")


def _cfg3(seed=3, nz=200, nx=200, nt=1500, nshot=16):
    """Autograd workload: linear v(z) 1500-2500 m/s, Gardner rho, 16 shots,
    200 receivers at z = 10 m, 12 Hz."""
    rng = np.random.default_rng(seed)
    dx = 10.0
    z = np.arange(nz, dtype=np.float64)[:, None] * np.ones((1, nx))
    vp = 1500.0 + 1000.0 * z / max(nz - 1, 1)
    rho = gardner_rho(vp)
    blobs, _ = gaussian_blobs(rng, (nz, nx), 6, 3.0, (-0.05, 0.05), 0.15 * nz, 0.85 * nz)
    blobs2, _ = gaussian_blobs(rng, (nz, nx), 6, 3.0, (-0.05, 0.05), 0.15 * nz, 0.85 * nz)
    dm = np.stack([blobs, blobs2])
    xs = [min(10 + 12 * k, nx - 1) for k in range(nshot)]
    geom = _surface_line_geometry(nz, nx, xs, [np.arange(nx)] * nshot, src_z=1, rec_z=1)
    dt = 1e-3
    return Workload("cfg3_2d_autograd", 2, nz, 1, nx, dx, dx, dx, dt, nt, 4, 20, 12.0,
                    vp, rho, dm, ricker(nt, dt, 12.0), geom, cg_iters=5,
                    notes="linear v(z), 6+6 Gaussian blobs")


def _cfg4(seed=4, nz=128, ny=256, nx=256, nt=3000, shots_per_side=4, rec_step=2):
    """3D dipping-layer LSRTM: 6 planar layers with dips <= 15 degrees,
    1800-3500 m/s, Gardner rho, 20 thin dipping reflectors in dm, 16 shots on a
    4x4 grid, receivers on every second surface cell."""
    rng = np.random.default_rng(seed)
    dx = 12.5
    z = np.arange(nz, dtype=np.float64)[:, None, None]
    y = np.arange(ny, dtype=np.float64)[None, :, None]
    x = np.arange(nx, dtype=np.float64)[None, None, :]
    nl = 6
    vl = np.linspace(1800.0, 3500.0, nl)
    depth0 = np.sort(rng.uniform(0.12 * nz, 0.9 * nz, size=nl - 1))
    layer = np.zeros((nz, ny, nx), dtype=np.int64)
    for d0 in depth0:
        dip = math.radians(rng.uniform(0, 15))
        az = rng.uniform(0, 2 * math.pi)
        surf = d0 + math.tan(dip) * ((x - nx / 2) * math.cos(az) + (y - ny / 2) * math.sin(az))
        layer += (z > surf).astype(np.int64)
    vp = vl[layer]
    rho = gardner_rho(vp)
    dm = np.zeros((2, nz, ny, nx))
    for _ in range(20):
        d0 = rng.uniform(0.1 * nz, 0.95 * nz)
        dip = math.radians(rng.uniform(0, 15))
        az = rng.uniform(0, 2 * math.pi)
        surf = d0 + math.tan(dip) * ((x - nx / 2) * math.cos(az) + (y - ny / 2) * math.sin(az))
        sheet = (np.abs(z - surf) < 0.5).astype(np.float64)
        for p in range(2):
            dm[p] += rng.uniform(-0.1, 0.1) * sheet
    s = shots_per_side
    pos = [int(round((i + 0.5) * nx / s)) for i in range(s)]
    posy = [int(round((i + 0.5) * ny / s)) for i in range(s)]
    src = []
    for iy in posy:
        for ix in pos:
            src.append(_flat(3, ny, nx, 1, iy, ix))
    ry, rx = np.meshgrid(np.arange(0, ny, rec_step), np.arange(0, nx, rec_step), indexing="ij")
    recs = _flat(3, ny, nx, 1, ry.ravel(), rx.ravel()).astype(np.int32)
    n = len(src)
    geom = Geometry(np.asarray(src, np.int32), np.arange(n + 1, dtype=np.int32) * recs.size,
                    np.tile(recs, n).astype(np.int32))
    dt = 1e-3
    return Workload("cfg4_3d_dipping", 3, nz, ny, nx, dx, dx, dx, dt, nt, 8, 20, 12.0,
                    vp, rho, dm, ricker(nt, dt, 12.0), geom, cg_iters=10,
                    notes="6 dipping layers 1800-3500 m/s, 20 thin reflectors")


def _cfg5(seed=5, nz=300, nx=2000, nt=3000, nshot=120, shot_dx=12, shot_x0=40,
          nrec_range=(120, 240), rec_dx=2, near=4, margin=100):
    """2D marine line, uneven batch: water layer (16 cells, 1500 m/s, rho 1000)
    over ~20 sediment layers 1500-3200 m/s, streamer receivers trailing +x with
    a seeded channel count per shot, aperture window = receiver span +- 100."""
    rng = np.random.default_rng(seed)
    dx = 12.5
    nw = 16
    vt = _layered_faulted(rng, nz - nw, nx, 20, 1550.0, 3200.0, 2, (2, 5), 0.02 * nz)
    vt = np.concatenate([np.full((nw, nx), 1500.0), vt], axis=0)
    rhot = gardner_rho(vt)
    rhot[:nw] = 1000.0
    v0 = vt.copy()
    r0 = rhot.copy()
    v0[nw:] = _smooth(vt[nw:], 8.0)
    r0[nw:] = _smooth(rhot[nw:], 8.0)
    dm = np.stack([np.log(vt) - np.log(v0), np.log(vt * rhot) - np.log(v0 * r0)])
    xs, recs, wx0, wnx = [], [], [], []
    for k in range(nshot):
        sx = min(shot_x0 + shot_dx * k, nx - 1)
        nr = int(rng.integers(nrec_range[0], nrec_range[1] + 1))
        rx = sx + near + rec_dx * np.arange(nr)
        rx = rx[rx < nx]
        xs.append(sx)
        recs.append(rx)
        lo = max(0, sx - margin)
        hi = min(nx, int(rx.max()) + margin + 1)
        wx0.append(lo)
        wnx.append(hi - lo)
    geom = _surface_line_geometry(nz, nx, xs, recs, src_z=1, rec_z=1)
    geom.win_x0 = np.asarray(wx0, np.int32)
    geom.win_nx = np.asarray(wnx, np.int32)
    dt = 1e-3
    return Workload("cfg5_2d_marine_uneven", 2, nz, 1, nx, dx, dx, dx, dt, nt, 8, 20, 20.0,
                    v0, r0, dm, ricker(nt, dt, 20.0), geom,
                    notes="water 200 m over 20 layers, streamer U[120,240] channels")


PRESETS = {1: _cfg1, 2: _cfg2, 3: _cfg3, 4: _cfg4, 5: _cfg5}


def preset(k: int, **overrides) -> Workload:
    """Workload preset k (1..5), seeded with k unless overridden."""
    return PRESETS[k](**overrides)


def small_case(ndim=2, nz=24, nx=30, ny=1, nt=120, order=4, npml=6, nshot=2, seed=11,
               dx=10.0, f0=25.0, dt=None, hetero=True, nrec=None) -> Workload:
    """A small random heterogeneous case used by tests: smooth random v and rho,
    random dm confined away from the interior edge, shots and receivers near
    the top."""
    rng = np.random.default_rng(seed)
    shape = (nz, nx) if ndim == 2 else (nz, ny, nx)
    if hetero:
        vp = 1800.0 + 400.0 * _smooth(rng.standard_normal(shape), 2.0) * 3
        rho = 1500.0 + 300.0 * _smooth(rng.standard_normal(shape), 2.0) * 3
    else:
        vp = np.full(shape, 2000.0)
        rho = np.full(shape, 1800.0)
    vp = np.clip(vp, 1400.0, 2600.0)
    rho = np.clip(rho, 1000.0, 2400.0)
    dm = rng.standard_normal((2,) + shape) * 0.05
    mask = np.zeros(shape)
    sl = tuple(slice(1, s - 1) for s in shape)
    mask[sl] = 1.0
    dm *= mask
    if dt is None:
        dt = 0.4 * dx / 2600.0 / math.sqrt(ndim)
    ny_ = ny if ndim == 3 else 1
    src, ptr, idx = [], [0], []
    for s in range(nshot):
        ix = int(rng.integers(1, nx - 1))
        iy = int(rng.integers(1, ny_ - 1)) if ndim == 3 else 0
        src.append(_flat(ndim, ny_, nx, 1, iy, ix))
        k = nrec if nrec is not None else int(rng.integers(3, 9))
        rz = rng.integers(0, nz, size=k)
        ry = rng.integers(0, ny_, size=k) if ndim == 3 else np.zeros(k, np.int64)
        rx = rng.integers(0, nx, size=k)
        idx.append(_flat(ndim, ny_, nx, rz, ry, rx))
        ptr.append(ptr[-1] + k)
    geom = Geometry(np.asarray(src, np.int32), np.asarray(ptr, np.int32),
                    np.concatenate(idx).astype(np.int32))
    return Workload("small", ndim, nz, ny_, nx, dx, dx, dx, dt, nt, order, npml, f0,
                    vp, rho, dm, ricker(nt, dt, f0), geom)


def image_pair(nz: int = 300, nx: int = 2000, seed: int = 5, nrefl: int = 40,
               noise: float = 0.01) -> tuple[np.ndarray, np.ndarray]:
    """A two-parameter image pair shaped like the marine-line workload's
    migrated image and its remigration, for the deblurring filters.

    m_rtm: [2, nz, nx] thin dipping reflectors with random amplitudes (the
    two planes share positions, different amplitudes). m_remig: each plane
    blurred by a Gaussian whose width grows with depth from 1 to 3 cells
    (the Hessian's resolution loss with depth), dimmed with depth, plus
    seeded white noise of relative size `noise`."""
    rng = np.random.default_rng(seed)
    zz = np.arange(nz, dtype=np.float64)[:, None]
    xx = np.arange(nx, dtype=np.float64)[None, :]
    m = np.zeros((2, nz, nx))
    for _ in range(nrefl):
        z0 = rng.uniform(0.05 * nz, 0.95 * nz)
        dip = rng.uniform(-0.15, 0.15)
        zl = z0 + dip * (xx - nx / 2)
        line = np.exp(-0.5 * ((zz - zl) / 0.6) ** 2)
        amps = rng.uniform(-0.1, 0.1, size=2)
        m[0] += amps[0] * line
        m[1] += amps[1] * line
    depth = zz / max(nz - 1, 1)
    remig = np.zeros_like(m)
    for q in range(2):
        b1 = _smooth(m[q], 1.0)
        b3 = _smooth(m[q], 3.0)
        remig[q] = ((1.0 - depth) * b1 + depth * b3) * (1.0 - 0.5 * depth)
        remig[q] += noise * np.abs(remig[q]).max() * rng.standard_normal((nz, nx))
    return m, remig


def psf_images(nz: int = 300, nx: int = 2000, spacing: int = 20, seed: int = 9,
               cross: float = 0.3) -> tuple[np.ndarray, np.ndarray]:
    """Synthetic PSF images shaped like the response of a spike comb (nodes at
    spacing//2 + k*spacing along both axes) for the two comb parameters.

    Returns (psf_vp, psf_ip), each [2, nz, nx]: around every node, plane q of
    the comb-in-parameter-j image holds a tilted, band-limited blob (a
    Mexican hat across a dipping axis times a Gaussian along it) whose width
    grows and amplitude falls with depth, with seeded per-node jitter of
    amplitude, width and tilt; off-diagonal planes (q != j) carry `cross`
    times an odd-symmetric blob. Values decay to ~1e-3 within spacing/2 of the
    node."""
    rng = np.random.default_rng(seed)
    zk = np.arange(spacing // 2, nz, spacing)
    xk = np.arange(spacing // 2, nx, spacing)
    out = [np.zeros((2, nz, nx)), np.zeros((2, nz, nx))]
    r = max(1, spacing // 2)
    dz, dx = np.meshgrid(np.arange(-r, r + 1, dtype=np.float64),
                         np.arange(-r, r + 1, dtype=np.float64), indexing="ij")
    for z in zk:
        depth = z / max(nz - 1, 1)
        for x in xk:
            for j in range(2):
                for q in range(2):
                    sig = (0.08 + 0.08 * depth) * spacing * rng.uniform(0.85, 1.15)
                    tilt = rng.uniform(-0.4, 0.4)
                    amp = (1.0 - 0.6 * depth) * rng.uniform(0.8, 1.2)
                    u = (dz * math.cos(tilt) + dx * math.sin(tilt)) / sig
                    v = (-dz * math.sin(tilt) + dx * math.cos(tilt)) / (2.0 * sig)
                    blob = (1.0 - u * u) * np.exp(-0.5 * (u * u + v * v))
                    if q != j:
                        blob = cross * u * np.exp(-0.5 * (u * u + v * v))
                    z0, z1 = max(0, z - r), min(nz, z + r + 1)
                    x0, x1 = max(0, x - r), min(nx, x + r + 1)
                    out[j][q, z0:z1, x0:x1] += amp * blob[z0 - z + r:z1 - z + r, x0 - x + r:x1 - x + r]
    return out[0], out[1]


def psf_images3(nz: int, ny: int, nx: int, spacing: int, seed: int = 9,
                cross: float = 0.3) -> tuple[np.ndarray, np.ndarray]:
    """3D counterpart of psf_images: (psf_vp, psf_ip), each [2, nz, ny, nx],
    a blob around every node of the 3D comb (a Mexican hat along a tilted
    axis in the z-x plane times Gaussians across it) with depth-dependent
    width and amplitude, seeded per-node jitter, and odd-symmetric
    cross-parameter responses."""
    rng = np.random.default_rng(seed)
    zk = np.arange(spacing // 2, nz, spacing)
    yk = np.arange(spacing // 2, ny, spacing)
    xk = np.arange(spacing // 2, nx, spacing)
    out = [np.zeros((2, nz, ny, nx)), np.zeros((2, nz, ny, nx))]
    r = max(1, spacing // 2)
    g = np.arange(-r, r + 1, dtype=np.float64)
    dz, dy, dx = np.meshgrid(g, g, g, indexing="ij")
    for z in zk:
        depth = z / max(nz - 1, 1)
        for y in yk:
            for x in xk:
                for j in range(2):
                    for q in range(2):
                        sig = (0.1 + 0.08 * depth) * spacing * rng.uniform(0.85, 1.15)
                        tilt = rng.uniform(-0.4, 0.4)
                        amp = (1.0 - 0.6 * depth) * rng.uniform(0.8, 1.2)
                        u = (dz * math.cos(tilt) + dx * math.sin(tilt)) / sig
                        v = (-dz * math.sin(tilt) + dx * math.cos(tilt)) / (2.0 * sig)
                        wy = dy / (2.0 * sig)
                        env = np.exp(-0.5 * (u * u + v * v + wy * wy))
                        blob = (1.0 - u * u) * env if q == j else cross * u * env
                        z0, z1 = max(0, z - r), min(nz, z + r + 1)
                        y0, y1 = max(0, y - r), min(ny, y + r + 1)
                        x0, x1 = max(0, x - r), min(nx, x + r + 1)
                        out[j][q, z0:z1, y0:y1, x0:x1] += amp * blob[z0 - z + r:z1 - z + r, y0 - y + r:y1 - y + r,
                                                                     x0 - x + r:x1 - x + r]
    return out[0], out[1]
