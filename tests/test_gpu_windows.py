"""Shots with uneven aperture windows in one launch, against the FP64 oracle.

Each shot runs on its own window's sub-model with its own CPML; shots of
different widths share the launches of a batch. Small marine-line cases
(ragged batches) check every record and image value; the marine-line
workload at full size (300 x 2000, 120 shots with windows of 440 to 680
columns, order 8, nt = 3000) checks sampled shots' records, a one-shot
migration after the full reverse time axis, and the FP32 dot test."""
import dataclasses

import numpy as np
import pytest

import lsrtm_inputs as li
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 1e-4


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def cpu(t):
    return t.detach().cpu().numpy().astype(np.float64)


def small_line(seed=5):
    w = li.preset(5, nz=36, nx=150, nt=300, nshot=5, shot_dx=26, shot_x0=8, nrec_range=(6, 20),
                  margin=9, seed=seed)
    return dataclasses.replace(w, npml=10)


def handle(w, **kw):
    from paper_2508_10405_gb300 import Lsrtm
    return Lsrtm.from_workload(w, **kw)


@pytest.mark.parametrize("batch", [0, 2])
def test_windowed_born_adjoint_hessian(batch):
    w = small_line()
    assert len(set(w.geom.win_nx.tolist())) > 1
    h = handle(w, shots_per_batch=batch)
    d = cpu(h.born(torch.tensor(w.dm, dtype=torch.float32, device="cuda")))
    ref = oracle.born(w, w.dm)
    print(f"windowed Born (batch {batch}): {rel(d, ref):.3e}")
    assert rel(d, ref) < TOL
    rng = np.random.default_rng(3)
    dres = rng.standard_normal(ref.shape)
    g, ph = h.adjoint(torch.tensor(dres, dtype=torch.float32, device="cuda"), pseudo_hessian=True)
    gref = oracle.adjoint(w, dres)
    print(f"windowed migration (batch {batch}): {rel(cpu(g), gref):.3e}")
    assert rel(cpu(g), gref) < TOL
    assert rel(cpu(ph), oracle.pseudo_hessian(w)) < TOL
    m = torch.tensor(rng.standard_normal((2,) + w.shape), dtype=torch.float32, device="cuda")
    Lm = h.born(m)
    a = float((Lm.double() ** 2).sum())
    b = float((m.double() * h.adjoint(Lm).double()).sum())
    print(f"windowed FP32 dot test: {abs(a - b) / a:.3e}")
    assert abs(a - b) / a < 1e-6
    h.close()


def test_full_width_windows_equal_plain_handle():
    w = small_line()
    wf = dataclasses.replace(w, geom=dataclasses.replace(
        w.geom, win_x0=np.zeros(w.geom.nshot, np.int32), win_nx=np.full(w.geom.nshot, w.nx, np.int32)))
    wp = dataclasses.replace(w, geom=dataclasses.replace(w.geom, win_x0=None, win_nx=None))
    dm = torch.tensor(w.dm, dtype=torch.float32, device="cuda")
    hf, hp = handle(wf), handle(wp)
    df, dp = hf.born(dm), hp.born(dm)
    gf, gp = hf.adjoint(dp), hp.adjoint(dp)
    print(f"full-width windows vs plain: records {rel(cpu(df), cpu(dp)):.3e}, images {rel(cpu(gf), cpu(gp)):.3e}")
    assert rel(cpu(df), cpu(dp)) < 1e-6 and rel(cpu(gf), cpu(gp)) < 1e-6
    hf.close()
    hp.close()


def test_window_geometry_errors():
    from paper_2508_10405_gb300 import LsrtmError, RECON_CHECKPOINT
    w = small_line()
    bad = dataclasses.replace(w, geom=dataclasses.replace(w.geom, win_x0=w.geom.win_x0 + 40))
    with pytest.raises(LsrtmError):
        handle(bad)   # receivers leave their windows (or windows leave the model)
    with pytest.raises(LsrtmError):
        handle(w, recon_mode=RECON_CHECKPOINT)


@pytest.fixture(scope="module")
def cfg5():
    w = li.preset(5)
    h = handle(w)
    yield w, h
    h.close()


def test_marine_line_full_size_records(cfg5):
    w, h = cfg5
    assert w.geom.win_nx.min() < w.geom.win_nx.max()
    d = h.born(torch.tensor(w.dm, dtype=torch.float32, device="cuda")).cpu().numpy()
    assert np.all(np.isfinite(d))
    ns = 400
    shots = [0, 61, 119]
    ref = oracle.born(w, w.dm, geom=w.geom.subset(shots), nt=ns)
    rows = np.concatenate([np.arange(w.geom.rec_ptr[s], w.geom.rec_ptr[s + 1]) for s in shots])
    e = rel(d[rows, :ns], ref)
    print(f"marine line full size, shots {shots}, first {ns} steps: {e:.3e}")
    assert e < TOL


def test_marine_line_full_size_migration_one_shot(cfg5):
    w, h = cfg5
    ns, s = 350, 77
    rng = np.random.default_rng(77)
    r0, r1 = w.geom.rec_ptr[s], w.geom.rec_ptr[s + 1]
    part = rng.standard_normal((r1 - r0, ns))
    dfull = torch.zeros((w.geom.nrec_total, w.nt), dtype=torch.float32, device="cuda")
    dfull[r0:r1, :ns] = torch.tensor(part, dtype=torch.float32, device="cuda")
    g = cpu(h.adjoint(dfull))
    ref = oracle.adjoint(w, part, geom=w.geom.subset([s]), nt=ns)
    e = rel(g, ref)
    print(f"marine line full size, migration of shot {s} after {w.nt - ns} reconstructed steps: {e:.3e}")
    assert e < TOL


def test_marine_line_full_size_dot(cfg5):
    w, h = cfg5
    rng = np.random.default_rng(8)
    m = torch.tensor(rng.standard_normal((2,) + w.shape), dtype=torch.float32, device="cuda")
    Lm = h.born(m)
    a = float((Lm.double() ** 2).sum())
    b = float((m.double() * h.adjoint(Lm).double()).sum())
    print(f"marine line full size FP32 dot test: {abs(a - b) / a:.3e}")
    assert abs(a - b) / a < 1e-6
