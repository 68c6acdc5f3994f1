"""Writes cfg2_cg_4shot.json: the FP64 oracle's CGNR on the 2D
Marmousi-shaped workload at its full grid (384 x 1152 interior, order 8,
nt = 4000) restricted to four of its shots, with seeded standard-normal data
(float32-representable, drawn by the same generator in the GPU test). Stores
the normalised misfits of iterations 0..3, the L2 norm of the final iterate
per parameter plane, and the iterate at 4096 seeded sample positions.

Calls only the oracle and the input generators. Run from the repository root:
    python tests/golden/make_cfg2_cg_golden.py
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import lsrtm_inputs as li  # noqa: E402
import oracle  # noqa: E402

SHOTS = [0, 31, 64, 95]
NITER = 3
DATA_SEED = 2024
SAMPLE_SEED = 2025
NSAMPLE = 4096


def case():
    w = li.preset(2)
    w.geom = w.geom.subset(SHOTS)
    d = np.random.default_rng(DATA_SEED).standard_normal((w.geom.nrec_total, w.nt)).astype(np.float32)
    idx = np.sort(np.random.default_rng(SAMPLE_SEED).choice(2 * w.nint, NSAMPLE, replace=False))
    return w, d, idx


def main():
    w, d, idx = case()
    t = time.time()
    x, mis = oracle.lsrtm_cg(w, d.astype(np.float64), NITER)
    out = {
        "what": "FP64 oracle CGNR, 2D Marmousi-shaped workload (384x1152, order 8, nt 4000), shots "
                f"{SHOTS}, seeded N(0,1) data (seed {DATA_SEED}), {NITER} iterations",
        "shots": SHOTS, "niter": NITER, "data_seed": DATA_SEED, "sample_seed": SAMPLE_SEED,
        "misfit": [float(v) for v in mis],
        "plane_norm": [float(np.linalg.norm(x[0])), float(np.linalg.norm(x[1]))],
        "sample_index": [int(i) for i in idx],
        "sample_value": [float(v) for v in x.reshape(-1)[idx]],
        "oracle_seconds": round(time.time() - t, 1),
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cfg2_cg_4shot.json")
    with open(path, "w") as f:
        json.dump(out, f)
    print(path, out["misfit"], out["oracle_seconds"])


if __name__ == "__main__":
    main()
