"""Pins of the oracle's per-shot aperture windows.

A windowed shot is modelled on its window's sub-model with its own CPML, so:
a window spanning the whole model is the plain operator (bit for bit); in a
laterally homogeneous medium with the perturbation inside the window, the
windowed records equal the unwindowed ones up to the CPML's residual
reflection; and the windowed L and L^T pass the dot test."""
import dataclasses

import numpy as np

import lsrtm_inputs as li
import oracle


def _line_case(hetero):
    w = li.small_case(nz=40, nx=90, nt=400, order=8, npml=12, nshot=1, seed=3, hetero=hetero,
                      dx=10.0, f0=20.0)
    src = np.array([1 * 90 + 30, 1 * 90 + 60], np.int32)
    recs = [1 * 90 + np.arange(25, 46), 1 * 90 + np.arange(55, 80)]
    ptr = np.array([0, recs[0].size, recs[0].size + recs[1].size], np.int32)
    w.geom = li.Geometry(src, ptr, np.concatenate(recs).astype(np.int32))
    dm = np.zeros((2, 40, 90))
    zz, xx = np.meshgrid(np.arange(40), np.arange(90), indexing="ij")
    dm[0] = 0.1 * np.exp(-((zz - 20) ** 2 + (xx - 35) ** 2) / 8.0)
    dm[1] = -0.05 * np.exp(-((zz - 22) ** 2 + (xx - 62) ** 2) / 8.0)
    return w, dm


def test_full_width_window_is_the_plain_operator():
    w, dm = _line_case(True)
    gw = dataclasses.replace(w.geom, win_x0=np.array([0, 0], np.int32), win_nx=np.array([90, 90], np.int32))
    d = oracle.born(w, dm)
    assert np.array_equal(oracle.born(w, dm, geom=gw), d)
    # images are the same per shot; only the order of the shot sum differs
    for got, ref in ((oracle.adjoint(w, d, geom=gw), oracle.adjoint(w, d)),
                     (oracle.pseudo_hessian(w, geom=gw), oracle.pseudo_hessian(w))):
        assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


def test_window_in_homogeneous_medium_matches_unwindowed():
    w, dm = _line_case(False)
    x0, nxw = np.array([10, 45], np.int32), np.array([50, 45], np.int32)
    gw = dataclasses.replace(w.geom, win_x0=x0, win_nx=nxw)
    win = oracle.born(w, dm, geom=gw)
    for s in range(2):
        dms = np.zeros_like(dm)
        dms[..., x0[s]:x0[s] + nxw[s]] = dm[..., x0[s]:x0[s] + nxw[s]]
        full = oracle.born(w, dms, geom=w.geom.subset([s]))
        rows = slice(w.geom.rec_ptr[s], w.geom.rec_ptr[s + 1])
        e = np.linalg.norm(win[rows] - full) / np.linalg.norm(full)
        assert e < 5e-3, (s, e)


def test_windowed_dot_product():
    w = li.preset(5, nz=36, nx=110, nt=260, nshot=4, shot_dx=22, shot_x0=8, nrec_range=(6, 14),
                  margin=9)
    w = dataclasses.replace(w, npml=10)
    assert np.any(w.geom.win_nx < w.nx) and len(set(w.geom.win_nx.tolist())) > 1
    rng = np.random.default_rng(4)
    m = rng.standard_normal((2,) + w.shape)
    d = rng.standard_normal((w.geom.nrec_total, w.nt))
    a = float(np.vdot(oracle.born(w, m), d))
    b = float(np.vdot(m, oracle.adjoint(w, d)))
    assert abs(a - b) <= 1e-12 * max(abs(a), abs(b))
