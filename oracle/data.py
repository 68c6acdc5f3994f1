"""FP64 oracle of the data-domain input: muted data residuals (Sec. 4).

TEST INFRASTRUCTURE ONLY (callers: tests/, smoke(), bench.py's CPU legs).

The data-domain inversion does not invert raw records: the observed data
(modelled in the true medium) minus the data modelled in the background
medium is multiplied by a muting mask that removes the direct arrivals and
the long-offset refractions (diving waves), leaving the near-offset
reflections. The paper shows the mask but does not define it; the reading
used here (and by the CUDA path) is a time-offset mask per receiver r and
recorded sample n:

  * offset o_r: horizontal distance between the shot's source and receiver r,
    sqrt(((ix_r - ix_s) dx)^2 + ((iy_r - iy_s) dy)^2) (metres);
  * time of sample n: t_n = (n + 1) dt (sample n holds p^{n+1});
  * direct-wave mute: t_d(r) = o_r / v_mute + t0, mask factor
    ramp(t_n - t_d(r), T_t);
  * far-offset mute: ramp(o_max - o_r, T_o) (no cut when o_max <= 0);
  * ramp(u, W) = 0 for u <= 0, 1 for u >= W, (1 - cos(pi u / W)) / 2 in
    between (W = 0: a hard step, 0 at u <= 0 and 1 above);
  * residual = mask * (d_obs - d_syn).
"""
from __future__ import annotations

import numpy as np


def ramp(u, width: float):
    """0 for u <= 0, 1 for u >= width, a raised-cosine rise in between."""
    u = np.asarray(u, np.float64)
    if width <= 0.0:
        return (u > 0.0).astype(np.float64)
    r = 0.5 * (1.0 - np.cos(np.pi * np.clip(u, 0.0, width) / width))
    return np.where(u <= 0.0, 0.0, np.where(u >= width, 1.0, r))


def offsets(w, geom=None) -> np.ndarray:
    """Horizontal source-receiver offset of every receiver row (metres)."""
    geom = w.geom if geom is None else geom
    ny = w.ny if w.ndim == 3 else 1
    out = np.zeros(geom.nrec_total)
    for s in range(geom.nshot):
        ks = int(geom.src_idx[s])
        xs, ys = ks % w.nx, (ks // w.nx) % ny
        for r in range(geom.rec_ptr[s], geom.rec_ptr[s + 1]):
            k = int(geom.rec_idx[r])
            xr, yr = k % w.nx, (k // w.nx) % ny
            out[r] = np.hypot((xr - xs) * w.dx, (yr - ys) * w.dy)
    return out


def mute_mask(w, v_mute: float, t0: float, t_taper: float, o_max: float, o_taper: float,
              geom=None, nt=None) -> np.ndarray:
    """Mask [nrec_total, nt] of the direct-wave and far-offset mutes."""
    nt = int(w.nt if nt is None else nt)
    o = offsets(w, geom)
    t = (np.arange(nt) + 1.0) * w.dt
    td = o / v_mute + t0
    mt = ramp(t[None, :] - td[:, None], t_taper)
    mo = np.ones_like(o) if o_max <= 0.0 else ramp(o_max - o, o_taper)
    return mt * mo[:, None]


def muted_residual(w, d_obs, d_syn, v_mute: float, t0: float, t_taper: float, o_max: float,
                   o_taper: float, geom=None) -> np.ndarray:
    """mask * (d_obs - d_syn); d_syn may be None (the mask applied to d_obs)."""
    d_obs = np.asarray(d_obs, np.float64)
    r = d_obs if d_syn is None else d_obs - np.asarray(d_syn, np.float64)
    return mute_mask(w, v_mute, t0, t_taper, o_max, o_taper, geom, d_obs.shape[1]) * r
