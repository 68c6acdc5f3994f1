"""The z-chunk autotuner (2D and fused 3D kernels): it picks one of the timed candidates, and the
operators give bit-identical results before and after (the chunking changes
which CTA computes a cell, not how)."""
import dataclasses

import numpy as np
import pytest

import lsrtm_inputs as li

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def handle(w, **kw):
    from paper_2508_10405_gb300 import Lsrtm
    return Lsrtm.from_workload(w, **kw)


def _check(w, **kw):
    h = handle(w, **kw)
    dm = torch.tensor(w.dm, dtype=torch.float32, device="cuda")
    d0 = h.born(dm).clone()
    g0 = h.adjoint(d0).clone()
    res = h.autotune(steps=6)
    print(f"{w.name} {kw}: chose tzc {res['tzc']} from {res['ms_per_step']}")
    assert res["tzc"] in res["ms_per_step"] and len(res["ms_per_step"]) >= 1
    assert all(v > 0 for v in res["ms_per_step"].values())
    d1 = h.born(dm)
    g1 = h.adjoint(d1)
    assert torch.equal(d0, d1) and torch.equal(g0, g1)
    h.close()


def test_autotune_2d_results_unchanged():
    _check(li.small_case(nz=70, nx=50, nt=120, order=8, npml=8, nshot=3, seed=301))
    _check(li.small_case(nz=90, nx=40, nt=100, order=4, npml=6, nshot=2, seed=302), shots_per_batch=1)


def test_autotune_windowed_and_checkpointed():
    from paper_2508_10405_gb300 import RECON_CHECKPOINT
    w = li.preset(5, nz=60, nx=150, nt=200, nshot=4, shot_dx=30, shot_x0=8, nrec_range=(6, 20), margin=9)
    _check(dataclasses.replace(w, npml=10))
    _check(li.small_case(nz=64, nx=40, nt=90, order=8, npml=6, nshot=2, seed=303),
           recon_mode=RECON_CHECKPOINT, checkpoint_interval=10)


def test_autotune_3d_results_unchanged():
    """The fused 3D kernels' z-chunk: several candidates, identical bits."""
    _check(li.small_case(ndim=3, nz=40, ny=14, nx=20, nt=40, order=4, npml=5, nshot=2, seed=304))
    _check(li.small_case(ndim=3, nz=44, ny=12, nx=18, nt=36, order=8, npml=6, nshot=2, seed=305))
