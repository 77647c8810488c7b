"""The oracle reproduces its committed regression values (tests/golden/oracle_regression.json,
written by tests/golden/make_golden.py from the oracle alone)."""
import json
import os

import numpy as np

import oracle
from paper_2203_07308_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "oracle_regression.json")


def test_oracle_regression_values():
    with open(GOLDEN) as f:
        gold = json.load(f)
    wl = synth.workloads()["c1_64"]
    g = wl.geom
    x = synth.phantom_batch(wl)[0]
    sino = oracle.project(g, 1, x)
    for v, j, val in gold["rays"]:
        assert abs(sino[v, j] - val) <= 1e-12 * max(1.0, abs(val))
    sino2 = oracle.project(g, 2, oracle.pool(x, 2), None, 1, 3)
    assert list(sino2.shape) == gold["sketch2_subset1of3_shape"]
    assert abs(sino2[0].sum() - gold["sketch2_subset1of3_row0_sum"]) < 1e-9
    z = x[20:36, 20:36] + 0.1 * synth.noise_draws((16, 16), 99)
    d = oracle.fgp(z, 0.02, 20)
    assert abs(d.sum() - gold["fgp20_patch_sum"]) < 1e-10
    assert abs(d[0, 0] - gold["fgp20_patch_00"]) < 1e-13
    L1, it1 = oracle.power_iter(g, 1, 100, 1e-7)
    assert abs(L1 - gold["power_L1"]) < 1e-9 * L1 and it1 == gold["power_L1_iters"]
    assert oracle.sample_count(g) == gold["samples_full"]
    w = synth.noise_draws((g.n_views, g.n_det), synth.noise_seed(wl.config_id))
    b = oracle.simulate(g, x, w, wl.noise_rel)
    stages = [synth.Stage(2, 2, 3), synth.Stage(1, 2, 1)]
    seq = synth.schedule_sequence(stages, 1)
    xr, log = oracle.pnp_run(g, stages, [1 / gold["power_L2"], 1 / gold["power_L1"]], seq, b,
                             alpha=1.0, lam=0.02, tv_iters=20, momentum=True, xt=x)
    assert np.abs(log - np.array(gold["pnp4_psnr"])).max() < 1e-9
    assert abs(xr.sum() - gold["pnp4_x_sum"]) < 1e-8
