"""The denoiser's last launch also writes the level-1 coefficient image of the
momentum point y when the next iteration is a full-grid mini-batch one; that
iteration then launches no coefficient-image kernel.  Both kernels build each
cell from the same four pixels of y with one shared formula, so a process with
PNP_FUSE_QUAD=0 (coefficient-image kernel in every iteration) must give the same
bits in x and y, and the PSNR log up to FP64 summation order, over schedules
that enter, leave and skip the fused path (sketched -> full grid, mini-batch ->
SVRG, empty stages, resumed runs), ragged and exact tilings, chained denoiser
launches, two classes in one call and a nine-image class (image-interleaved
coefficient images).
Parity with the oracle is checked by the run suites, which use the fused path."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SCRIPT = r"""
import sys, numpy as np, torch
sys.path.insert(0, ROOT)
import paper_2203_07308_gb300 as pnp
from paper_2203_07308_gb300 import synth

def problem(n, views, det, batch, seed):
    g = synth.make_geometry(n, views, det, batch=batch)
    rng = np.random.default_rng(seed)
    xt = np.stack([synth.ellipse_phantom(n, seed + k) for k in range(batch)]).astype(np.float32)
    b = rng.poisson(50.0, size=(batch, views, det)).astype(np.float32) * 0.01
    return g, torch.from_numpy(xt).cuda(), torch.from_numpy(b).cuda()

out = {}
# one class: ragged 16-pixel tiles (n = 100), 25 denoiser iterations (three launches),
# an odd iteration count, an empty stage and a y output
g, xt, b = problem(100, 48, 128, 2, 3)
plan = pnp.Plan(g)
plan.set_launch_shapes(tile=16)
st = [synth.Stage(2, 3, 4), synth.Stage(4, 0, 1), synth.Stage(1, 6, 4)]
seq = synth.schedule_sequence(st, 5)
x = torch.zeros(2, 100, 100, device="cuda")
y = torch.zeros_like(x)
logs = pnp.run_many([dict(plan=plan, stages=st, eta=[2e-4, 1e-4, 1e-4], seq=seq, b=b, x=x, xtrue=xt, y=y)],
                    lam=0.01, tv_iters=25)
out["x1"], out["y1"], out["p1"] = x.cpu().numpy(), y.cpu().numpy(), logs[0]
# resumed from iteration 4 of the same schedule
x4, y4 = torch.zeros_like(x), torch.zeros_like(x)
pnp.run_many([dict(plan=plan, stages=[synth.Stage(2, 3, 4), synth.Stage(1, 1, 4)], eta=[2e-4, 1e-4],
                   seq=seq[:4], b=b, x=x4, y=y4)], lam=0.01, tv_iters=25)
pnp.run_many([dict(plan=plan, stages=st, eta=[2e-4, 1e-4, 1e-4], seq=seq, b=b, x=x4, y=y4, start_iter=4)],
             lam=0.01, tv_iters=25)
out["x4"] = x4.cpu().numpy()
# two classes in one call: default and 22-pixel tiles, mini-batch -> SVRG -> mini-batch, no momentum
ga, xa, ba = problem(64, 40, 96, 2, 7)
gb, xb, bb = problem(88, 36, 112, 1, 9)
pa, pb_ = pnp.Plan(ga), pnp.Plan(gb)
pb_.set_launch_shapes(tile=22)
sa = [synth.Stage(1, 3, 5), synth.Stage(1, 4, 5, estimator=1), synth.Stage(1, 2, 5)]
sb = [synth.Stage(2, 2, 3), synth.Stage(1, 5, 3)]
xa_ = torch.zeros(2, 64, 64, device="cuda")
xb_ = torch.zeros(1, 88, 88, device="cuda")
logs = pnp.run_many([dict(plan=pa, stages=sa, eta=[1e-4] * 3, seq=synth.schedule_sequence(sa, 11), b=ba, x=xa_,
                          xtrue=xa),
                     dict(plan=pb_, stages=sb, eta=[2e-4, 1e-4], seq=synth.schedule_sequence(sb, 12), b=bb,
                          x=xb_, xtrue=xb)], lam=0.02, tv_iters=12, momentum=False)
out["xa"], out["xb"], out["pa"], out["pb"] = xa_.cpu().numpy(), xb_.cpu().numpy(), logs[0], logs[1]
# nine images: image-interleaved coefficient images, written by the denoiser for the 2x and full levels
gc, xc, bc = problem(48, 24, 64, 9, 13)
pc = pnp.Plan(gc)
pc.set_launch_shapes(tile=16)
sc = [synth.Stage(2, 3, 3), synth.Stage(1, 3, 2)]
xc_ = torch.zeros(9, 48, 48, device="cuda")
logs = pnp.run_many([dict(plan=pc, stages=sc, eta=[2e-4, 1e-4], seq=synth.schedule_sequence(sc, 14), b=bc,
                          x=xc_, xtrue=xc)], lam=0.02, tv_iters=12)
out["xc"], out["pc"] = xc_.cpu().numpy(), logs[0]
np.savez(sys.argv[1], **out)
"""


def test_fused_coefficient_image_changes_no_bit(tmp_path):
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2203_07308_gb300 import build
    build.build()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = tmp_path / "run.py"
    script.write_text(SCRIPT.replace("ROOT", repr(root)))
    res = []
    for fuse in ("1", "0"):
        out = tmp_path / f"o{fuse}.npz"
        env = dict(os.environ, PNP_FUSE_QUAD=fuse)
        subprocess.run([sys.executable, str(script), str(out)], env=env, check=True, timeout=900)
        res.append(np.load(out))
    assert sorted(res[0].files) == sorted(res[1].files)
    for k in res[0].files:
        assert np.isfinite(res[0][k]).all(), k
        if k.startswith("p"):
            # the FP64 squared-error sums visit the tile's pixels in another thread
            # order when the region carries the ring: equal up to that rounding
            np.testing.assert_allclose(res[0][k], res[1][k], rtol=1e-12, atol=0, err_msg=k)
        else:
            assert np.array_equal(res[0][k], res[1][k]), k
    # the resumed run reaches the same iterate as the uninterrupted one
    assert np.array_equal(res[0]["x4"], res[0]["x1"])
