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
against FP64 central differences along random directions. J is quadratic,
so its central difference along u is exactly <L dm - d, L u>, which the
oracle evaluates in FP64."""
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


def test_autograd_gradient_vs_fp64_central_differences():
    """50 random directions on a reduced autograd-shaped case (100 x 100, 4
    shots, nt = 600): <grad, u> against the FP64 central difference of J,
    which for the quadratic J is exactly <L dm - d, L u> (one oracle Born
    modelling per direction)."""
    w = li.preset(3, nz=100, nx=100, nt=600, nshot=4)
    rng = np.random.default_rng(33)
    d_obs = oracle.born(w, w.dm)
    x = 0.5 * w.dm
    grad = _grad_gpu(w, x, d_obs)
    r = oracle.born(w, x) - d_obs
    errs = []
    for _ in range(50):
        u = rng.standard_normal(x.shape)
        cd = float(np.vdot(r, oracle.born(w, u)))
        errs.append(abs(float(np.vdot(grad, u)) - cd) / (np.linalg.norm(grad) * np.linalg.norm(u)))
    print(f"autograd vs FP64 central differences, 50 directions: max {max(errs):.3e}")
    assert max(errs) < 1e-5, max(errs)
