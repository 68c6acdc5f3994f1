"""The non-finite guard: NaN injected on the host (into the observed data or
the model perturbation) is found inside the time loop, the rest of the loop
is skipped, and the call fails with LSRTM_ERR_NONFINITE naming the loop and
the step; the handle stays usable. Nothing here faults the device: the NaN
is ordinary input data, and every kernel stays in bounds."""
import numpy as np
import pytest

import lsrtm_inputs as li

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

NONFINITE = 5

CASE2 = dict(nz=37, nx=45, nt=300, order=4, npml=8, nshot=3, seed=31)
CASE3 = dict(ndim=3, nz=12, ny=10, nx=14, nt=70, order=4, npml=5, nshot=2, seed=213)


def handle(w, **kw):
    from paper_2508_10405_gb300 import Lsrtm
    return Lsrtm.from_workload(w, **kw)


def dev(a):
    return torch.tensor(np.asarray(a), dtype=torch.float32, device="cuda")


def nan_dm(w):
    dm = np.array(w.dm, np.float32)
    idx = tuple(s // 2 for s in dm.shape[1:])
    dm[(0,) + idx] = np.nan
    return dm


def expect_nonfinite(fn, *words):
    from paper_2508_10405_gb300 import LsrtmError
    with pytest.raises(LsrtmError) as ei:
        fn()
    assert ei.value.status == NONFINITE, str(ei.value)
    for wd in words:
        assert wd in str(ei.value), str(ei.value)
    return str(ei.value)


@pytest.mark.parametrize("interval,step", [(0, 63), (10, 9)])
def test_born_guard_names_the_step(interval, step):
    """NaN in dm makes dp NaN from step 0 (NaN times the zero background);
    the first check after it is the interval's last step."""
    w = li.small_case(**CASE2)
    h = handle(w, guard_interval=interval)
    clean = h.born(dev(w.dm)).cpu().numpy()
    h.born(dev(nan_dm(w)))
    expect_nonfinite(h.synchronize, "Born", f"step {step};")
    again = h.born(dev(w.dm)).cpu().numpy()
    h.synchronize()
    assert np.array_equal(again, clean)


def test_guard_off_lets_nan_through():
    w = li.small_case(**CASE2)
    h = handle(w, guard_interval=-1)
    d = h.born(dev(nan_dm(w))).cpu().numpy()
    h.synchronize()
    assert not np.isfinite(d).all()


@pytest.mark.parametrize("kw", [{}, {"plan": 1}, {"recon_mode": 1, "checkpoint_interval": 40}],
                         ids=["batched", "plain", "checkpoint"])
def test_nan_in_observed_data_ends_cgnr(kw):
    """NaN in the last sample of one trace enters lambda_p at the first
    reverse step; the migration loop of lsrtm_cg_begin trips the guard at
    reverse step 63 (time step nt - 64), and the solve stops one iteration
    later instead of running its 10."""
    w = li.small_case(**CASE2)
    h = handle(w, **kw)
    d = h.born(dev(w.dm))
    bad = d.clone()
    bad[1, w.nt - 1] = float("nan")
    expect_nonfinite(lambda: h.cg_solve(bad, 10), "migration", f"step {w.nt - 64};")
    assert h.cg_get_state()["iter"] <= 2
    x, mis = h.cg_solve(d, 3)
    x_ref, mis_ref = handle(w, **kw).cg_solve(d, 3)
    assert np.array_equal(x.cpu().numpy(), x_ref.cpu().numpy())
    assert np.array_equal(mis, mis_ref)


def test_nan_scalar_in_resumed_state_ends_cgnr():
    """A NaN planted in a saved search direction (restored through
    lsrtm_cg_set_state) trips the guard in the next Born loop."""
    w = li.small_case(**CASE2)
    h = handle(w)
    d = h.born(dev(w.dm))
    h.cg_begin(d)
    h.cg_iterate(1)
    st = h.cg_get_state()
    st["p"][0, 5, 5] = np.nan
    h.cg_set_state(st)
    expect_nonfinite(lambda: h.cg_iterate(3, misfit=True), "Born")


def test_3d_guard():
    w = li.small_case(**CASE3)
    h = handle(w, guard_interval=8)
    clean = h.born(dev(w.dm)).cpu().numpy()
    h.born(dev(nan_dm(w)))
    expect_nonfinite(h.synchronize, "Born", "step 7;")
    d = dev(clean)
    bad = d.clone()
    bad[0, w.nt - 1] = float("nan")
    expect_nonfinite(lambda: h.cg_solve(bad, 4), "migration", f"step {w.nt - 8};")
    again = h.born(dev(w.dm)).cpu().numpy()
    h.synchronize()
    assert np.array_equal(again, clean)
