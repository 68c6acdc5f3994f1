"""Per-iteration JSON logging of a CGNR / PCGNR solve (Sec. 3).

Each iteration writes one JSON line: the normalised misfit ||r_k|| / ||d||
(the convergence measure of the paper's figures), the relative model error
||x_k - m|| / ||m|| when the true perturbation m is known, the wall seconds
of the iteration, and per time-loop kind the device milliseconds (CUDA
events on the library's stream), the cell-update rate and the algorithmic
HBM bandwidth. The solve is the library's step-wise CGNR, one
lsrtm_cg_iterate call per iteration, so its iterates are the ones
lsrtm_cg_solve returns, bit for bit.

`Lsrtm.cg_solve` routes through here when the environment variable
LSRTM_PROFILE names a file (appended to) or is "-" (stderr)."""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

# Algorithmic HBM bytes per cell update (FP32, one pass per step, model read
# raw): Born = 2 x (3 + 3) state fields read + written + 4 model arrays;
# migration = 6 state fields read + written + 2 model arrays + 2 image planes
# read + written; background only = p and the velocities read + written +
# dt kappa and 1/rho.
BYTES_PER_CELL = {("born", 2): 64.0, ("adjoint", 2): 72.0, ("born", 3): 80.0, ("adjoint", 3): 88.0,
                  ("background", 2): 32.0, ("background", 3): 40.0}


def _sink(dest):
    if dest is None:
        return None, False
    if hasattr(dest, "write"):
        return dest, False
    if dest == "-":
        return sys.stderr, False
    return open(dest, "a"), True


def iteration_record(op, k: int, misfit: float, seconds: float, timings: dict, model_error=None) -> dict:
    """One log line from lsrtm_timing_read's per-kind sums of an iteration."""
    rec = {"event": "cg_iteration", "iteration": k, "misfit": misfit, "seconds": seconds}
    if model_error is not None:
        rec["rel_model_error"] = model_error
    ms_all, cells_all, bytes_all = 0.0, 0.0, 0.0
    for kind in ("born", "background", "adjoint"):
        ms, cells = timings[f"{kind}_ms"], timings[f"{kind}_cells"]
        if ms <= 0:
            continue
        b = BYTES_PER_CELL[(kind, op.ndim)] * cells
        rec[kind] = {"ms": ms, "gcell_per_s": cells / ms / 1e6, "gb_per_s": b / ms / 1e6,
                     "launches": int(timings[f"{kind}_launches"])}
        ms_all, cells_all, bytes_all = ms_all + ms, cells_all + cells, bytes_all + b
    if ms_all > 0:
        rec["gcell_per_s"] = cells_all / ms_all / 1e6
        rec["gb_per_s"] = bytes_all / ms_all / 1e6
    return rec


def cg_solve_logged(op, d, niter: int, x0=None, precond=False, param_mask=3, log=None, m_true=None):
    """CGNR through the step-wise API with one JSON line per iteration to
    `log` (a path, "-" for stderr, or a file object). Returns (x, misfits)
    like Lsrtm.cg_solve."""
    out, close = _sink(log)
    mt = None if m_true is None else np.asarray(m_true.detach().cpu() if hasattr(m_true, "detach") else m_true,
                                                np.float64)
    try:
        op.timing(True)
        op.timings(reset=True)
        t0 = time.perf_counter()
        op.cg_begin(d, x0=x0, precond=precond, param_mask=param_mask)
        x, m0 = op.cg_result()
        tm = op.timings(reset=True)
        mis = [m0]

        def err(x):
            if mt is None:
                return None
            return float(np.linalg.norm(x.cpu().numpy().astype(np.float64) - mt) / np.linalg.norm(mt))

        if out is not None:
            out.write(json.dumps(iteration_record(op, 0, m0, time.perf_counter() - t0, tm, err(x))) + "\n")
        for k in range(1, niter + 1):
            t0 = time.perf_counter()
            m = float(op.cg_iterate(1, misfit=True)[0])
            sec = time.perf_counter() - t0
            tm = op.timings(reset=True)
            mis.append(m)
            if out is not None:
                e = err(op.cg_result()[0]) if mt is not None else None
                out.write(json.dumps(iteration_record(op, k, m, sec, tm, e)) + "\n")
                out.flush()
        x, _ = op.cg_result()
        return x, np.array(mis)
    finally:
        op.timing(False)
        if close:
            out.close()


def env_log():
    """The LSRTM_PROFILE destination, or None."""
    v = os.environ.get("LSRTM_PROFILE", "")
    return v or None
