"""Writes cfg3_autograd.json for the autograd workload (200 x 200, order 4,
nt = 1500, 16 shots) at its full size, from the FP64 oracle only:

  * CGNR: three iterations on seeded standard-normal data (float32
    representable): normalised misfits, plane norms of the iterate and the
    iterate at 2048 seeded sample positions;
  * central differences: J(x) = 1/2 ||L x - d||^2 with x = dm / 2 of the
    workload and the same data; J is quadratic, so its central difference
    along u is exactly <L x - d, L u>, stored for 50 seeded directions u
    (float32 representable, N(0, 1)).

Run from the repository root:  python tests/golden/make_cfg3_golden.py
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

DATA_SEED = 303
SAMPLE_SEED = 304
DIR_SEED = 305
NITER = 3
NDIR = 50
NSAMPLE = 2048


def case():
    w = li.preset(3)
    d = np.random.default_rng(DATA_SEED).standard_normal((w.geom.nrec_total, w.nt)).astype(np.float32)
    x = (0.5 * w.dm).astype(np.float32)
    idx = np.sort(np.random.default_rng(SAMPLE_SEED).choice(2 * w.nint, NSAMPLE, replace=False))
    return w, d, x, idx


def directions(w):
    rng = np.random.default_rng(DIR_SEED)
    for _ in range(NDIR):
        yield rng.standard_normal((2,) + tuple(w.shape)).astype(np.float32)


def main():
    w, d, x, idx = case()
    t = time.time()
    xc, mis = oracle.lsrtm_cg(w, d.astype(np.float64), NITER)
    r = oracle.born(w, x.astype(np.float64)) - d.astype(np.float64)
    cd = [float(np.vdot(r, oracle.born(w, u.astype(np.float64)))) for u in directions(w)]
    out = {
        "what": "FP64 oracle, autograd workload (200x200, order 4, nt 1500, 16 shots): CGNR on seeded "
                f"N(0,1) data (seed {DATA_SEED}), and central differences <L x - d, L u> of "
                "J = 1/2 ||L x - d||^2 at x = dm/2 along seeded directions",
        "data_seed": DATA_SEED, "sample_seed": SAMPLE_SEED, "dir_seed": DIR_SEED,
        "niter": NITER, "misfit": [float(v) for v in mis],
        "plane_norm": [float(np.linalg.norm(xc[0])), float(np.linalg.norm(xc[1]))],
        "sample_index": [int(i) for i in idx],
        "sample_value": [float(v) for v in xc.reshape(-1)[idx]],
        "central_difference": cd,
        "oracle_seconds": round(time.time() - t, 1),
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cfg3_autograd.json")
    with open(path, "w") as f:
        json.dump(out, f)
    print(path, out["misfit"], out["oracle_seconds"])


if __name__ == "__main__":
    main()
