"""3D operators through the C ABI against the FP64 oracle.

Small grids (both orders, several shots, ragged extents) for Born, migration,
the FP32 dot tests, the pseudo-Hessian, PSF, CGNR and 16-bit bands; and the 3D
dipping-layer workload at its full grid size (296 x 296 x 168 padded cells,
order 8, nt = 3000) on two of its shots with BF16 bands: Born records over the
first steps against the oracle, and the FP32 dot test over the whole time
axis."""
import numpy as np
import pytest

import lsrtm_inputs as li
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 1e-4

CASES3 = {
    "o4": dict(ndim=3, nz=14, ny=11, nx=17, nt=90, order=4, npml=5, nshot=2, seed=131),
    "o8": dict(ndim=3, nz=13, ny=12, nx=15, nt=80, order=8, npml=6, nshot=3, seed=132),
}


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def cpu(t):
    return t.detach().cpu().numpy().astype(np.float64)


def handle(w, **kw):
    from paper_2508_10405_gb300 import Lsrtm
    return Lsrtm.from_workload(w, **kw)


@pytest.fixture(scope="module", params=sorted(CASES3))
def case3(request):
    return request.param, li.small_case(**CASES3[request.param])


def test_3d_born_and_migration(case3):
    name, w = case3
    h = handle(w)
    d = cpu(h.born(torch.tensor(w.dm, dtype=torch.float32, device="cuda")))
    ref = oracle.born(w, w.dm)
    print(f"3D Born {name}: rel L2 {rel(d, ref):.3e}")
    assert rel(d, ref) < TOL
    rng = np.random.default_rng(5)
    dres = rng.standard_normal(ref.shape)
    g = cpu(h.adjoint(torch.tensor(dres, dtype=torch.float32, device="cuda")))
    gref = oracle.adjoint(w, dres)
    print(f"3D migration {name}: rel L2 {rel(g, gref):.3e}")
    assert rel(g, gref) < TOL


def test_3d_dot_fp32(case3):
    name, w = case3
    h = handle(w)
    rng = np.random.default_rng(6)
    m = torch.tensor(rng.standard_normal((2,) + w.shape), dtype=torch.float32, device="cuda")
    Lm = h.born(m).double()
    a = float((Lm * Lm).sum())
    b = float((m.double() * h.adjoint(Lm.float()).double()).sum())
    print(f"3D FP32 dot test {name}: {abs(a - b) / a:.3e}")
    assert abs(a - b) / a < 1e-6


def test_3d_pseudo_hessian_psf_and_cg():
    w = li.small_case(**CASES3["o8"])
    h = handle(w)
    rng = np.random.default_rng(2)
    d = torch.tensor(rng.standard_normal((w.geom.nrec_total, w.nt)), dtype=torch.float32, device="cuda")
    _, ph = h.adjoint(d, pseudo_hessian=True)
    assert rel(cpu(ph), oracle.pseudo_hessian(w)) < TOL
    for param in (0, 1):
        assert rel(cpu(h.psf(param, 4)), oracle.psf(w, param, 4)) < TOL
    dobs = oracle.born(w, w.dm)
    x, mis = h.cg_solve(torch.tensor(dobs, dtype=torch.float32, device="cuda"), 3)
    xr, misr = oracle.lsrtm_cg(w, dobs, 3)
    print(f"3D CGNR: misfit max abs diff {np.max(np.abs(mis - misr)):.3e}, iterate rel L2 {rel(cpu(x), xr):.3e}")
    assert np.all(np.abs(mis - misr) < TOL), (mis, misr)
    assert rel(cpu(x), xr) < TOL


BAND_CASES = {
    # the tiny grid: its 5-cell pad and M-deep bands are most of the volume, so
    # the BF16 rounding of the bands (2^-9 relative) reaches the image almost
    # undamped; the error is stated and bounded, not held to the 1e-3 bar
    "tiny": dict(ndim=3, nz=14, ny=11, nx=17, nt=90, order=4, npml=5, nshot=2, seed=131),
    # a larger grid, bands still a visible share of the volume (the 1e-3
    # bar of the mixed-precision path is held at the workload's full size,
    # test_3d_full_size_two_shots)
    "mid": dict(ndim=3, nz=40, ny=36, nx=44, nt=220, order=8, npml=10, nshot=2, seed=133),
}


@pytest.mark.parametrize("fmt,case,tol", [("bf16", "tiny", 5e-3), ("fp16", "tiny", 1e-3),
                                          ("bf16", "mid", 3e-3), ("fp16", "mid", 1e-3)])
def test_3d_16bit_bands(fmt, case, tol):
    from paper_2508_10405_gb300 import BAND_BF16, BAND_FP16
    w = li.small_case(**BAND_CASES[case])
    rng = np.random.default_rng(3)
    dres = rng.standard_normal((w.geom.nrec_total, w.nt))
    dt = torch.tensor(dres, dtype=torch.float32, device="cuda")
    g32 = cpu(handle(w).adjoint(dt))
    g16 = cpu(handle(w, band_precision=BAND_BF16 if fmt == "bf16" else BAND_FP16).adjoint(dt))
    ref = oracle.adjoint(w, dres)
    print(f"3D {fmt} bands, {case} grid: {rel(g16, ref):.3e} vs oracle, {rel(g16, g32):.3e} vs FP32 bands")
    assert rel(g16, ref) < tol
    assert rel(g16, g32) < tol


def test_3d_full_size_two_shots():
    """Full 3D grid, order 8, nt = 3000, shots 0 and 5 of the dipping-layer
    workload. A Gaussian scatterer 4 cells below each source makes the first
    60 steps carry a real Born arrival (the workload's reflectors are reached
    later; before that the exact records are numerical precursors of order
    1e-34, below FP32's normal range)."""
    from paper_2508_10405_gb300 import BAND_BF16
    w = li.preset(4)
    w.geom = w.geom.subset([0, 5])
    dm = w.dm.copy()
    zz, yy, xx = np.meshgrid(*[np.arange(n, dtype=np.float64) for n in w.shape], indexing="ij")
    for s in w.geom.src_idx:
        sx = s % w.nx
        sy = (s // w.nx) % w.ny
        sz = s // (w.nx * w.ny)
        r2 = (zz - sz - 4) ** 2 + (yy - sy) ** 2 + (xx - sx) ** 2
        dm[0] += 0.05 * np.exp(-r2 / 4.0)
        dm[1] -= 0.05 * np.exp(-r2 / 4.0)
    h = handle(w)
    d = h.born(torch.tensor(dm, dtype=torch.float32, device="cuda"))
    ns = 60
    ref = oracle.born(w, dm, nt=ns)
    got = cpu(d)[:, :ns]
    print(f"3D full-size Born, first {ns} steps: rel L2 {rel(got, ref):.3e}")
    assert rel(got, ref) < TOL
    rng = np.random.default_rng(8)
    m = torch.tensor(rng.standard_normal((2,) + w.shape), dtype=torch.float32, device="cuda")
    Lm = h.born(m)
    a = float((Lm.double() ** 2).sum())
    g32 = h.adjoint(Lm)
    b = float((m.double() * g32.double()).sum())
    print(f"3D full-size FP32 dot test: {abs(a - b) / a:.3e}")
    assert abs(a - b) / a < 1e-6
    h.close()
    h16 = handle(w, band_precision=BAND_BF16)
    g16 = h16.adjoint(Lm)
    e16 = rel(cpu(g16), cpu(g32))
    print(f"3D full-size migration with BF16 bands vs FP32 bands: rel L2 {e16:.3e}")
    assert e16 < 1e-3
    h16.close()


def test_3d_full_size_migration_vs_oracle():
    """Full 3D grid, order 8, nt = 3000, one shot of the dipping-layer
    workload: the residual is zero except in the first n_s samples, so L^T d
    equals the oracle's L^T of that shot with nt = n_s; on the GPU the
    background is first rebuilt from the boundary bands through all of the
    3000 - n_s later steps, which tests the 3D reconstruction over the full
    time axis. A Gaussian scatterer below the source gives the early
    background field a clear image to compare."""
    w = li.preset(4)
    w.geom = w.geom.subset([5])
    ns = 40
    rng = np.random.default_rng(44)
    nrec = w.geom.nrec_total
    part = rng.standard_normal((nrec, ns))
    h = handle(w)
    dfull = torch.zeros((nrec, w.nt), dtype=torch.float32, device="cuda")
    dfull[:, :ns] = torch.tensor(part, dtype=torch.float32, device="cuda")
    g = cpu(h.adjoint(dfull))
    h.close()
    ref = oracle.adjoint(w, part, nt=ns)
    print(f"3D full-size migration, residual in the first {ns} of {w.nt} steps: rel L2 {rel(g, ref):.3e}")
    assert rel(g, ref) < TOL
