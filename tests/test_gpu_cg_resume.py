"""Save and resume of a step-wise CGNR solve (the Krylov driver of Sec. 3).

Four uninterrupted iterations against two iterations, a state saved to an
.npz file, a fresh handle that begins the same solve, restores the state and
runs two more: the iterate and the misfit history must be bit-identical
(plain and preconditioned, both parameters and mono-parameter Ip)."""
import numpy as np
import pytest

import lsrtm_inputs as li

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("precond,mask", [(False, 3), (True, 3), (False, 2)])
def test_resume_is_bitwise(tmp_path, precond, mask):
    from paper_2508_10405_gb300 import Lsrtm, LsrtmError
    w = li.small_case(nz=30, nx=44, nt=220, order=8, npml=8, nshot=3, seed=17, nrec=24)
    dm = torch.tensor(w.dm, dtype=torch.float32, device="cuda")
    h1 = Lsrtm.from_workload(w)
    d = h1.born(dm)
    h1.cg_begin(d, precond=precond, param_mask=mask)
    mis_ref = h1.cg_iterate(4, misfit=True)
    x_ref, _ = h1.cg_result()

    h2 = Lsrtm.from_workload(w)
    h2.cg_begin(d, precond=precond, param_mask=mask)
    h2.cg_iterate(2)
    st = h2.cg_get_state()
    assert st["iter"] == 2
    np.savez(tmp_path / "cg.npz", **st)
    h2.close()

    h3 = Lsrtm.from_workload(w)
    with pytest.raises(LsrtmError, match="ERR_STATE"):
        h3.cg_set_state(st)                      # no active solve yet
    h3.cg_begin(d, precond=precond, param_mask=mask)
    loaded = dict(np.load(tmp_path / "cg.npz"))
    h3.cg_set_state(loaded)
    mis = h3.cg_iterate(2, misfit=True)
    x, _ = h3.cg_result()
    assert torch.equal(x, x_ref)
    assert np.array_equal(mis, mis_ref[2:])
    assert h3.cg_get_state()["iter"] == 4
    h1.close()
    h3.close()
