"""Per-iteration JSON logging of CGNR: the logged solve runs step-wise and
returns the iterates of lsrtm_cg_solve bit for bit; each line carries the
misfit, the relative model error and the loop rates."""
import io
import json

import numpy as np
import pytest

import lsrtm_inputs as li

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_logged_cg_matches_cg_solve():
    from paper_2508_10405_gb300 import Lsrtm
    w = li.small_case(nz=37, nx=45, nt=300, order=4, npml=8, nshot=3, seed=31)
    dm = torch.tensor(w.dm, dtype=torch.float32, device="cuda")
    h = Lsrtm.from_workload(w)
    d = h.born(dm)
    x_ref, mis_ref = Lsrtm.from_workload(w).cg_solve(d, 4)
    buf = io.StringIO()
    x, mis = h.cg_solve(d, 4, log=buf, m_true=w.dm)
    assert np.array_equal(x.cpu().numpy(), x_ref.cpu().numpy())
    assert np.array_equal(mis, mis_ref)
    lines = [json.loads(s) for s in buf.getvalue().splitlines()]
    assert [r["iteration"] for r in lines] == list(range(5))
    assert [r["misfit"] for r in lines] == list(mis)
    assert lines[0]["rel_model_error"] == pytest.approx(1.0)
    assert lines[-1]["rel_model_error"] < lines[0]["rel_model_error"]
    for r in lines[1:]:
        assert r["born"]["gcell_per_s"] > 0 and r["adjoint"]["gcell_per_s"] > 0
        assert r["gb_per_s"] > 0 and r["seconds"] > 0
