"""The free surface (method of images on the first interior row) through the
C ABI against the FP64 oracle: Born records and migration images within the
FP32 bar of 1e-4, the FP32 dot test within 1e-6, receivers on the surface row
recording zero, 2D and 3D, both orders, boundary-band and checkpoint
reconstruction, the pseudo-Hessian; a source on the surface row is refused."""
import dataclasses

import numpy as np
import pytest

import lsrtm_inputs as li
import oracle
from lsrtm_inputs import Geometry

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 1e-4


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def cpu(t):
    return t.detach().cpu().numpy().astype(np.float64)


def fs_case(**kw):
    w = dataclasses.replace(li.small_case(**kw), free_surface=True)
    idx = w.geom.rec_idx.copy()
    idx[0] = idx[0] % (w.nx * w.ny)   # one receiver on the surface row
    return dataclasses.replace(w, geom=Geometry(w.geom.src_idx, w.geom.rec_ptr, idx))


CASES = {
    "2d_o4": dict(nz=37, nx=45, nt=300, order=4, npml=8, nshot=3, seed=231),
    "2d_o8": dict(nz=41, nx=53, nt=260, order=8, npml=10, nshot=2, seed=232),
    "3d_o4": dict(ndim=3, nz=14, ny=13, nx=17, nt=90, order=4, npml=5, nshot=2, seed=233),
    "3d_o8": dict(ndim=3, nz=16, ny=12, nx=15, nt=80, order=8, npml=6, nshot=2, seed=234),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_free_surface_born_adjoint_dot(name):
    from paper_2508_10405_gb300 import Lsrtm
    w = fs_case(**CASES[name])
    h = Lsrtm.from_workload(w)
    d = cpu(h.born(torch.tensor(w.dm, dtype=torch.float32, device="cuda")))
    ref = oracle.born(w, w.dm)
    assert np.all(d[0] == 0.0) and np.all(ref[0] == 0.0)   # surface receiver
    rng = np.random.default_rng(11)
    dres = rng.standard_normal(ref.shape)
    g = cpu(h.adjoint(torch.tensor(dres, dtype=torch.float32, device="cuda")))
    gref = oracle.adjoint(w, dres)
    m = torch.tensor(rng.standard_normal((2,) + w.shape), dtype=torch.float32, device="cuda")
    Lm = h.born(m).double()
    a = float((Lm * Lm).sum())
    b = float((m.double() * h.adjoint(Lm.float()).double()).sum())
    h.synchronize()
    h.close()
    print(f"free surface {name}: Born {rel(d, ref):.3e}, migration {rel(g, gref):.3e}, dot {abs(a - b) / a:.3e}")
    assert rel(d, ref) < TOL
    assert rel(g, gref) < TOL
    assert abs(a - b) / a < 1e-6


@pytest.mark.parametrize("name", ["2d_o8", "3d_o4"])
def test_free_surface_checkpoint_equals_boundary(name):
    """Checkpointed reconstruction repeats the boundary mode's arithmetic:
    the same images bit for bit, with the free surface."""
    from paper_2508_10405_gb300 import RECON_BOUNDARY, RECON_CHECKPOINT, Lsrtm
    w = fs_case(**CASES[name])
    rng = np.random.default_rng(12)
    dres = torch.tensor(rng.standard_normal((w.geom.nrec_total, w.nt)), dtype=torch.float32, device="cuda")
    hb = Lsrtm.from_workload(w, recon_mode=RECON_BOUNDARY)
    hc = Lsrtm.from_workload(w, recon_mode=RECON_CHECKPOINT, checkpoint_interval=17)
    gb, gc = hb.adjoint(dres), hc.adjoint(dres)
    assert torch.equal(gb, gc)
    hb.close()
    hc.close()


def test_free_surface_pseudo_hessian():
    from paper_2508_10405_gb300 import Lsrtm
    w = fs_case(**CASES["2d_o4"])
    h = Lsrtm.from_workload(w)
    _, ph = h.adjoint(torch.zeros((w.geom.nrec_total, w.nt), dtype=torch.float32, device="cuda"),
                      pseudo_hessian=True)
    assert rel(cpu(ph), oracle.pseudo_hessian(w)) < TOL
    h.close()


def test_free_surface_refuses_surface_source():
    from paper_2508_10405_gb300 import Lsrtm, LsrtmError
    w = fs_case(**CASES["2d_o4"])
    src = w.geom.src_idx.copy()
    src[0] = src[0] % w.nx
    bad = dataclasses.replace(w, geom=Geometry(src, w.geom.rec_ptr, w.geom.rec_idx))
    with pytest.raises(LsrtmError, match="ERR_GEOMETRY"):
        Lsrtm.from_workload(bad)
