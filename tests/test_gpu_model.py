"""Nonlinear modelling and muted data residuals (Sec. 4) on the GPU against
the FP64 oracle.

* lsrtm_model: 2D orders 4 and 8, 3D, aperture windows (uneven widths in one
  batch): records within 1e-4 of the oracle's;
* the GPU's own linearisation: (F(m0 + eps dm) - F(m0)) / eps against its
  Born records, with the same error as the oracle's (the two operators of the
  GPU path are consistent with each other, not just with the oracle);
* lsrtm_mute_residual: device and host buffers, with and without the
  background data, every sample against the oracle's mask (FP64 mute times);
* the whole input pipeline (true-model and background handles, residual,
  mute) against the oracle's;
* argument errors."""
import dataclasses

import numpy as np
import pytest

import lsrtm_inputs as li
import oracle
from oracle import data as od

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _h(w, **kw):
    from paper_2508_10405_gb300 import Lsrtm
    return Lsrtm.from_workload(w, **kw)


@pytest.mark.parametrize("case", ["2d_o4", "2d_o8", "3d_o8", "windows"])
def test_model_matches_the_oracle(case):
    if case == "2d_o4":
        w = li.small_case(nz=40, nx=70, nt=300, order=4, npml=10, nshot=3, seed=21, nrec=30)
    elif case == "2d_o8":
        w = li.small_case(nz=45, nx=90, nt=350, order=8, npml=12, nshot=2, seed=22, nrec=40)
    elif case == "3d_o8":
        w = li.small_case(ndim=3, nz=20, ny=22, nx=24, nt=120, order=8, npml=8, nshot=2, seed=23, nrec=30)
    else:
        w = li.preset(5, nz=36, nx=110, nt=260, nshot=4, shot_dx=22, shot_x0=8, nrec_range=(6, 14), margin=9)
        w = dataclasses.replace(w, npml=10)
        assert len(set(w.geom.win_nx.tolist())) > 1
    h = _h(w)
    got = h.model().double().cpu().numpy()
    ref = oracle.model(w)
    e = rel(got, ref)
    print(f"{case}: model records {e:.3e}")
    assert e < 1e-4
    h.close()


def test_linearisation_of_the_gpu_operators():
    w = li.small_case(nz=30, nx=40, nt=200, order=8, npml=8, nshot=2, seed=5, nrec=25)
    vmax = float(np.max(w.vp)) * 1.05
    eps = 0.1   # numerator 3% of |eps L dm|, well above the FP32 noise of the records
    vp = w.vp * np.exp(eps * w.dm[0])
    rho = w.rho * np.exp(eps * (w.dm[1] - w.dm[0]))
    h0 = _h(w, pml_vmax=vmax)
    h1 = _h(dataclasses.replace(w, vp=vp, rho=rho), pml_vmax=vmax)
    F0 = h0.model().double().cpu().numpy()
    F1 = h1.model().double().cpu().numpy()
    Ldm = h0.born(torch.tensor(w.dm, dtype=torch.float32, device="cuda")).double().cpu().numpy()
    e_gpu = np.linalg.norm(F1 - F0 - eps * Ldm) / np.linalg.norm(eps * Ldm)
    R0 = oracle.model(w, vmax=vmax)
    R1 = oracle.model(w, vp=vp, rho=rho, vmax=vmax)
    RL = oracle.born(w, w.dm, vmax=vmax)
    e_orc = np.linalg.norm(R1 - R0 - eps * RL) / np.linalg.norm(eps * RL)
    print(f"linearisation error: GPU {e_gpu:.5e}, oracle {e_orc:.5e}")
    assert abs(e_gpu - e_orc) <= 0.05 * e_orc
    h0.close()
    h1.close()


def _line(nt=600):
    nx = 161
    w = li.small_case(nz=60, nx=nx, nt=nt, order=8, npml=20, nshot=2, seed=3, hetero=False, dx=10.0, f0=20.0)
    w.geom = li.Geometry(np.array([1 * nx + 50, 1 * nx + 110], np.int32), np.array([0, nx, 2 * nx], np.int32),
                         np.concatenate([1 * nx + np.arange(nx)] * 2).astype(np.int32))
    return w


@pytest.mark.parametrize("host", [False, True])
@pytest.mark.parametrize("with_syn", [False, True])
def test_mute_residual_every_sample(host, with_syn):
    w = _line(nt=500)
    rng = np.random.default_rng(1)
    d_obs = rng.standard_normal((w.geom.nrec_total, w.nt)).astype(np.float32)
    d_syn = rng.standard_normal((w.geom.nrec_total, w.nt)).astype(np.float32) if with_syn else None
    args = (2000.0, 0.1, 0.0125, 600.0, 150.0)
    h = _h(w)
    if host:
        from paper_2508_10405_gb300 import binding
        out = np.zeros_like(d_obs)
        rc = h._lib.lsrtm_mute_residual(h._h, binding._ptr(d_obs), None if d_syn is None else binding._ptr(d_syn),
                                        *args, binding._ptr(out))
        assert rc == 0
        got = out.astype(np.float64)
    else:
        dd = torch.tensor(d_obs, device="cuda")
        ds = None if d_syn is None else torch.tensor(d_syn, device="cuda")
        got = h.mute_residual(dd, ds, *args).double().cpu().numpy()
    ref = od.muted_residual(w, d_obs.astype(np.float64), None if d_syn is None else d_syn.astype(np.float64), *args)
    assert np.max(np.abs(got - ref)) <= 2e-6 * np.max(np.abs(ref))
    # the mute decision (t_n after the mute time, offset inside the cut) is
    # taken in FP64 on both sides: every sample the oracle zeroes is zero
    assert np.all(got[od.mute_mask(w, *args) == 0.0] == 0.0)
    h.close()


def test_hard_mute_and_in_place():
    w = _line(nt=300)
    d = torch.ones((w.geom.nrec_total, w.nt), device="cuda")
    h = _h(w)
    h.mute_residual(d, None, 1800.0, 0.02, 0.0, 0.0, 0.0, out=d)       # in place, step mute, no offset cut
    ref = od.mute_mask(w, 1800.0, 0.02, 0.0, 0.0, 0.0)
    assert np.array_equal(d.cpu().numpy().astype(np.float64), ref)
    h.close()


def test_mute_times_outside_the_record():
    """Mute times past the record mute every sample (a vanishing v_mute mutes
    every receiver but the zero-offset ones, whose mute time is t0); one long
    before it mutes none (the taper has ended at the first sample)."""
    w = _line(nt=120)
    d = torch.ones((w.geom.nrec_total, w.nt), device="cuda")
    h = _h(w)
    for v_mute, t0 in ((2000.0, 1e300), (2000.0, 10.0)):
        assert torch.count_nonzero(h.mute_residual(d, None, v_mute, t0, 0.01)).item() == 0
    got = h.mute_residual(d, None, 1e-300, 0.0, 0.01).double().cpu().numpy()
    ref = od.mute_mask(w, 1e-300, 0.0, 0.01, 0.0, 0.0)
    assert np.all(got[ref == 0.0] == 0.0) and np.max(np.abs(got - ref)) < 1e-6
    assert np.all(got[od.offsets(w) > 0.0] == 0.0)
    assert torch.equal(h.mute_residual(d, None, 2000.0, -1e300, 0.01), d)
    h.close()


def test_input_pipeline_against_the_oracle():
    w = _line()
    vp2, rho2 = w.vp.copy(), w.rho.copy()
    vp2[30:], rho2[30:] = 2600.0, 2100.0
    vmax = 2600.0
    args = (2000.0, 2.0 / 20.0, 0.25 / 20.0, 500.0, 100.0)
    h_bg = _h(w, pml_vmax=vmax)
    h_true = _h(dataclasses.replace(w, vp=vp2, rho=rho2), pml_vmax=vmax)
    d_obs = h_true.model()
    d_bg = h_bg.model()
    res = h_bg.mute_residual(d_obs, d_bg, *args).double().cpu().numpy()
    ref = od.muted_residual(w, oracle.model(w, vp=vp2, rho=rho2, vmax=vmax), oracle.model(w, vmax=vmax), *args)
    e = rel(res, ref)
    print(f"muted residual: {e:.3e}")
    assert e < 1e-3      # a difference of two records of similar size: FP32 modelling error amplified
    h_bg.close()
    h_true.close()


def test_argument_errors():
    from paper_2508_10405_gb300 import LsrtmError
    w = _line(nt=50)
    h = _h(w)
    d = torch.zeros((w.geom.nrec_total, w.nt), device="cuda")
    for args in ((0.0, 0.1, 0.01, 0.0, 0.0), (2000.0, 0.1, -1.0, 0.0, 0.0), (2000.0, 0.1, 0.01, 100.0, -1.0),
                 (2000.0, float("nan"), 0.01, 0.0, 0.0)):
        with pytest.raises(LsrtmError):
            h.mute_residual(d, None, *args)
    h.close()
