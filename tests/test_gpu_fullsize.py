"""Parity at the benchmark's full size and launch configuration.

The 2D Marmousi-shaped workload (384 x 1152 interior, order 8, nt = 4000,
96 shots, all shots in one batch exactly as bench.py runs it) on the GPU,
against the FP64 oracle on sampled outputs the oracle computes one by one:

  * Born records: the first n_s time samples of sampled shots (records up to
    step n_s do not depend on later steps), oracle run with nt = n_s;
  * migration: residual zero except the first n_s samples of one shot, so
    L^T d equals the oracle's L^T on that shot with nt = n_s; on the GPU the
    background is rebuilt from the boundary bands through every one of the
    4000 - n_s later steps before the residual starts, which tests the
    reconstruction over the full time axis;
  * FP32 dot test <L m, L m> = <m, L^T L m> on the full workload.

The autograd workload (200 x 200, 16 shots, nt = 1500): the gradient of
J = 1/2 ||L dm - d||^2 through torch.autograd (backward = L^T on the GPU)
against FP64 central differences along 50 seeded directions (J is
quadratic, so its central difference along u is exactly <L dm - d, L u>),
and LSRTM by a torch CG loop over the autograd Function. The FP64 values for
the full-size CG and difference checks are too slow for the oracle inside a
test run; they are stored in tests/golden/ by scripts that call only the
oracle."""
import json
import os

import numpy as np
import pytest

import lsrtm_inputs as li
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 1e-4
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def cfg2():
    from paper_2508_10405_gb300 import Lsrtm
    w = li.preset(2)
    h = Lsrtm.from_workload(w)
    yield w, h
    h.close()


def test_born_full_size_sampled_shots(cfg2):
    w, h = cfg2
    dm = torch.tensor(w.dm, dtype=torch.float32, device="cuda")
    d = h.born(dm).cpu().numpy()
    ns = 320
    shots = [0, 47, 95]
    geom = w.geom.subset(shots)
    ref = oracle.born(w, w.dm, geom=geom, nt=ns)
    rows = np.concatenate([np.arange(w.geom.rec_ptr[s], w.geom.rec_ptr[s + 1]) for s in shots])
    got = d[rows, :ns]
    assert np.all(np.isfinite(d))
    print(f"full-size Born, shots {shots}, first {ns} steps: rel L2 {rel(got, ref):.3e}")
    assert rel(got, ref) < TOL, rel(got, ref)


def test_adjoint_full_size_one_shot_residual(cfg2):
    w, h = cfg2
    ns = 260
    s = 60
    rng = np.random.default_rng(60)
    r0, r1 = w.geom.rec_ptr[s], w.geom.rec_ptr[s + 1]
    part = rng.standard_normal((r1 - r0, ns))
    dfull = torch.zeros((w.geom.nrec_total, w.nt), dtype=torch.float32, device="cuda")
    dfull[r0:r1, :ns] = torch.tensor(part, dtype=torch.float32, device="cuda")
    g = h.adjoint(dfull).cpu().numpy()
    ref = oracle.adjoint(w, part, geom=w.geom.subset([s]), nt=ns)
    print(f"full-size migration, shot {s}, residual in the first {ns} of {w.nt} steps: rel L2 {rel(g, ref):.3e}")
    assert rel(g, ref) < TOL, rel(g, ref)


def test_dot_product_full_size(cfg2):
    w, h = cfg2
    rng = np.random.default_rng(7)
    m = torch.tensor(rng.standard_normal((2,) + w.shape), dtype=torch.float32, device="cuda")
    Lm = h.born(m)
    a = float((Lm.double() ** 2).sum())
    b = float((m.double() * h.adjoint(Lm).double()).sum())
    print(f"full-size FP32 dot test: {abs(a - b) / a:.3e}")
    assert abs(a - b) / a < 1e-6, (a, b)


def test_bf16_bands_full_size(cfg2):
    """The mixed-precision bar at the benchmark's size: the migration image
    with BF16 bands (one FP32 scale per band per step) within relative L2
    1e-3 of the FP32-band image, for the data L dm of the workload."""
    from paper_2508_10405_gb300 import BAND_BF16, Lsrtm
    w, h = cfg2
    dm = torch.tensor(w.dm, dtype=torch.float32, device="cuda")
    d = h.born(dm)
    g32 = h.adjoint(d).double().cpu().numpy()
    h16 = Lsrtm.from_workload(w, band_precision=BAND_BF16)
    g16 = h16.adjoint(d).double().cpu().numpy()
    h16.close()
    e = rel(g16, g32)
    print(f"full-size migration, BF16 vs FP32 bands: rel L2 {e:.3e}")
    assert e < 1e-3, e


def _grad_gpu(w, x, d_obs):
    from paper_2508_10405_gb300 import Lsrtm, born_op
    h = Lsrtm.from_workload(w)
    BornOp = born_op()
    xt = torch.tensor(x, dtype=torch.float32, device="cuda", requires_grad=True)
    dt = torch.tensor(d_obs, dtype=torch.float32, device="cuda")
    J = 0.5 * ((BornOp.apply(xt, h) - dt) ** 2).sum()
    J.backward()
    g = xt.grad.double().cpu().numpy()
    h.close()
    return g


def test_autograd_gradient_full_size_vs_oracle():
    """Autograd workload at full size: the GPU gradient of J equals the FP64
    oracle's L^T (L dm - d)."""
    w = li.preset(3)
    d_obs = oracle.born(w, w.dm)
    x = 0.5 * w.dm
    grad = _grad_gpu(w, x, d_obs)
    ref = oracle.adjoint(w, oracle.born(w, x) - d_obs)
    print(f"autograd gradient vs FP64 oracle: rel L2 {rel(grad, ref):.3e}")
    assert rel(grad, ref) < TOL, rel(grad, ref)


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _sampled_rel(x, gold):
    """Relative L2 distance of an iterate from the oracle's at its stored
    sample positions, and the largest relative error of the plane norms."""
    xs = x.reshape(-1)[np.asarray(gold["sample_index"])]
    ref = np.asarray(gold["sample_value"])
    en = max(abs(np.linalg.norm(x[i]) - gold["plane_norm"][i]) / gold["plane_norm"][i] for i in range(2))
    return rel(xs, ref), en


def test_autograd_gradient_vs_fp64_central_differences():
    """Autograd workload at full size (200 x 200, 16 shots, nt = 1500): the
    gradient of J = 1/2 ||L x - d||^2 through torch.autograd (backward = L^T
    on the GPU) along 50 seeded directions u against the FP64 central
    difference of J, which for the quadratic J is exactly <L x - d, L u>
    (tests/golden/cfg3_autograd.json, written by make_cfg3_golden.py from
    the oracle)."""
    gold = _golden("cfg3_autograd.json")
    w = li.preset(3)
    d = np.random.default_rng(gold["data_seed"]).standard_normal((w.geom.nrec_total, w.nt)).astype(np.float32)
    x = (0.5 * w.dm).astype(np.float32)
    grad = _grad_gpu(w, x, d)
    rng = np.random.default_rng(gold["dir_seed"])
    errs = []
    for cd in gold["central_difference"]:
        u = rng.standard_normal((2,) + tuple(w.shape)).astype(np.float32).astype(np.float64)
        errs.append(abs(float(np.vdot(grad, u)) - cd) / (np.linalg.norm(grad) * np.linalg.norm(u)))
    print(f"autograd vs FP64 central differences, {len(errs)} directions: max {max(errs):.3e}")
    assert len(errs) == 50
    assert max(errs) < 1e-5, max(errs)


def _torch_cgls(h, d, niter):
    """CGNR (CGLS form, Sec. 3) written as a plain torch loop over the
    autograd Function: L p is BornOp.apply, L^T r is the gradient of
    <L p, r> taken by torch.autograd (whose backward is the library's
    migration)."""
    from paper_2508_10405_gb300 import born_op
    BornOp = born_op()

    def L(m):
        return BornOp.apply(m, h)

    def LT(r):
        m = torch.zeros((2,) + h.shape, dtype=torch.float32, device="cuda", requires_grad=True)
        (g,) = torch.autograd.grad(L(m), m, grad_outputs=r)
        return g

    x = torch.zeros((2,) + h.shape, dtype=torch.float32, device="cuda")
    r = d.clone()
    s = LT(r)
    p = s.clone()
    gamma = float((s.double() ** 2).sum())
    dn = float(d.double().norm())
    mis = [float(r.double().norm()) / dn]
    with torch.no_grad():
        for _ in range(niter):
            q = h.born(p)
            alpha = gamma / float((q.double() ** 2).sum())
            x += alpha * p
            r -= alpha * q
            with torch.enable_grad():
                s = LT(r)
            gnew = float((s.double() ** 2).sum())
            p = s + (gnew / gamma) * p
            gamma = gnew
            mis.append(float(r.double().norm()) / dn)
    return x, np.asarray(mis)


def test_lsrtm_by_torch_cg_over_autograd_function():
    """LSRTM of the autograd workload at full size by a torch CG loop over
    the autograd Function: equal to the library's own CGNR and to the FP64
    oracle's CGNR (misfits and the iterate at stored sample positions, from
    tests/golden/cfg3_autograd.json) within 1e-4."""
    from paper_2508_10405_gb300 import Lsrtm
    gold = _golden("cfg3_autograd.json")
    w = li.preset(3)
    d = np.random.default_rng(gold["data_seed"]).standard_normal((w.geom.nrec_total, w.nt)).astype(np.float32)
    dt = torch.tensor(d, device="cuda")
    h = Lsrtm.from_workload(w)
    xt, mist = _torch_cgls(h, dt, gold["niter"])
    xl, misl = h.cg_solve(dt, gold["niter"])
    h.close()
    xt, xl = xt.double().cpu().numpy(), xl.double().cpu().numpy()
    es, en = _sampled_rel(xt, gold)
    print(f"torch CG over the Function: vs library CGNR rel L2 {rel(xt, xl):.3e}, misfits vs oracle "
          f"{np.max(np.abs(mist - gold['misfit'])):.3e}, samples vs oracle {es:.3e}, plane norms {en:.3e}")
    assert rel(xt, xl) < TOL
    assert np.max(np.abs(mist - np.asarray(gold["misfit"]))) < TOL
    assert np.max(np.abs(misl - np.asarray(gold["misfit"]))) < TOL
    assert es < TOL and en < TOL


def test_cg_config2_grid_four_shots_vs_oracle():
    """Three CGNR iterations on the 2D Marmousi-shaped workload at its full
    grid and time axis (384 x 1152, order 8, nt = 4000) on four of its
    shots, against the FP64 oracle's CGNR stored in
    tests/golden/cfg2_cg_4shot.json: misfits within 1e-4 absolute, the
    iterate within 1e-4 relative L2 at 4096 seeded sample positions and in
    its plane norms."""
    from paper_2508_10405_gb300 import Lsrtm
    gold = _golden("cfg2_cg_4shot.json")
    w = li.preset(2)
    w.geom = w.geom.subset(gold["shots"])
    d = np.random.default_rng(gold["data_seed"]).standard_normal((w.geom.nrec_total, w.nt)).astype(np.float32)
    h = Lsrtm.from_workload(w)
    x, mis = h.cg_solve(torch.tensor(d, device="cuda"), gold["niter"])
    h.close()
    x = x.double().cpu().numpy()
    es, en = _sampled_rel(x, gold)
    em = np.max(np.abs(mis - np.asarray(gold["misfit"])))
    print(f"config-2 grid CGNR, shots {gold['shots']}: misfits {em:.3e}, samples {es:.3e}, plane norms {en:.3e}")
    assert em < TOL and es < TOL and en < TOL
