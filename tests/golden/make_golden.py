"""Writes ``oracle_regression.json``: a few small oracle outputs stored as text.

The values are produced by the FP64 oracle only (``oracle/``) on seeded inputs
from ``paper_2203_07308_gb300.synth``; nothing here touches the CUDA path.  The
test suite re-runs the oracle and compares, so an accidental change to the
oracle's arithmetic shows up as a diff to this file in review.

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2203_07308_gb300 import synth  # noqa: E402

RAYS = [(0, 30), (0, 47), (13, 50), (45, 60), (89, 40)]


def main():
    wl = synth.workloads()["c1_64"]
    g = wl.geom
    x = synth.phantom_batch(wl)[0]
    sino = oracle.project(g, 1, x)
    sino2 = oracle.project(g, 2, oracle.pool(x, 2), None, 1, 3)
    z = x[20:36, 20:36] + 0.1 * synth.noise_draws((16, 16), 99)
    L1, it1 = oracle.power_iter(g, 1, 100, 1e-7)
    w = synth.noise_draws((g.n_views, g.n_det), synth.noise_seed(wl.config_id))
    b = oracle.simulate(g, x, w, wl.noise_rel)
    seq = synth.schedule_sequence([synth.Stage(2, 2, 3), synth.Stage(1, 2, 1)], 1)
    L2, _ = oracle.power_iter(g, 2, 100, 1e-7)
    xr, log = oracle.pnp_run(g, [synth.Stage(2, 2, 3), synth.Stage(1, 2, 1)], [1 / L2, 1 / L1],
                             seq, b, alpha=1.0, lam=0.02, tv_iters=20, momentum=True, xt=x)
    out = {
        "_note": "FP64 oracle outputs on the 64x64 / 90 views x 96 bins workload; written by make_golden.py",
        "rays": [[v, j, float(sino[v, j])] for v, j in RAYS],
        "sketch2_subset1of3_row0_sum": float(sino2[0].sum()),
        "sketch2_subset1of3_shape": list(sino2.shape),
        "fgp20_patch_sum": float(oracle.fgp(z, 0.02, 20).sum()),
        "fgp20_patch_00": float(oracle.fgp(z, 0.02, 20)[0, 0]),
        "power_L1": L1,
        "power_L1_iters": it1,
        "power_L2": L2,
        "pnp4_psnr": [float(v) for v in log],
        "pnp4_x_sum": float(xr.sum()),
        "samples_full": oracle.sample_count(g),
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_regression.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
