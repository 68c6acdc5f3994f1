"""The shot-parallel CGNR / PCGNR driver over the real CUDA operator (one
rank, no process group): equal to the FP64 oracle's CGNR and PCGNR within
1e-4. The multi-rank exchange itself is tested over gloo ranks on CPU."""
import numpy as np
import pytest

import lsrtm_inputs as li
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 1e-4


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.mark.parametrize("precond", [False, True])
def test_shot_parallel_cg_over_gpu_handle(precond):
    from paper_2508_10405_gb300 import Lsrtm
    from paper_2508_10405_gb300.distributed import ShotParallelCG, pcg_diagonal
    w = li.small_case(nz=30, nx=36, nt=220, order=8, npml=9, nshot=3, seed=301)
    d = oracle.born(w, w.dm)
    h = Lsrtm.from_workload(w)
    minv = pcg_diagonal(h) if precond else None
    x, mis = ShotParallelCG(h).solve(torch.tensor(d, dtype=torch.float32, device="cuda"), 3, precond=minv)
    xr, misr = oracle.lsrtm_cg(w, d, 3, precond=precond)
    e = rel(x.double().cpu().numpy(), xr)
    print(f"ShotParallelCG over Lsrtm (precond={precond}): misfits {np.max(np.abs(np.asarray(mis) - misr)):.3e}, "
          f"iterate {e:.3e}")
    assert np.max(np.abs(np.asarray(mis) - misr)) < TOL
    assert e < TOL
    h.close()
