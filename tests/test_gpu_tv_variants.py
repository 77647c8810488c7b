"""The FGP denoiser variants inside Algorithm 1 against the FP64 oracle: the
shared-memory tiles, the register-resident warp tiles (tile = 1) and strips
(tile = 2, 3, 4), pinned
with pnp_set_launch_shapes, on ragged and uneven sizes, with iteration counts
that split unevenly over launches, and with the PSNR log (per-tile partials)."""
import numpy as np
import pytest

import oracle
import paper_2203_07308_gb300 as pnp
from paper_2203_07308_gb300 import build, synth

pytestmark = pytest.mark.gpu
TOL_RECON = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    pnp.load()


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


@pytest.mark.parametrize("tile", [1, 2, 3, 4, 16, 22])
@pytest.mark.parametrize("n,views,det,batch,tv_iters", [(64, 60, 96, 2, 20), (37, 24, 60, 3, 7),
                                                       (100, 40, 150, 1, 3), (48, 30, 72, 2, 11)])
def test_denoiser_variants_in_algorithm1(tile, n, views, det, batch, tv_iters):
    g = synth.make_geometry(n, views, det, batch=batch)
    plan = pnp.Plan(g)
    plan.set_launch_shapes(tile=tile)
    x = np.stack([f32(synth.ellipse_phantom(n, 70 + i, (4, 7))) for i in range(batch)])
    rng = np.random.default_rng(n)
    b = f32(np.stack([oracle.project(g, 1, xi) for xi in x]) + 0.3 * rng.standard_normal((batch, views, det)))
    stages = [synth.Stage(1, 4, 3)]
    seq = synth.schedule_sequence(stages, 2)
    eta = [0.8 / oracle.power_iter(g, 1, 60, 1e-7)[0]]
    d_x = dev(np.zeros((batch, n, n)))
    log = plan.run(stages, eta, seq, dev(b), d_x, alpha=0.8, lam=0.05, tv_iters=tv_iters, xtrue=dev(x))
    got = host(d_x)
    for i in range(batch):
        xr, lr = oracle.pnp_run(g, stages, eta, seq, b[i], None, alpha=0.8, lam=0.05, tv_iters=tv_iters, xt=x[i])
        assert rel(got[i], xr) < TOL_RECON, (i, rel(got[i], xr))
        assert np.abs(log[:, i] - lr).max() < 1e-3


def test_mixed_classes_with_different_denoiser_variants():
    """run_many: one class tuned to the warp tiles, another to shared-memory
    tiles, a third to strips, in one call (the classes then share the
    shared-memory tiles); all against the oracle."""
    import torch
    specs = [(synth.make_geometry(64, 60, 96, batch=2), 1), (synth.make_geometry(48, 40, 72, batch=1), 16),
             (synth.make_geometry(80, 40, 120, batch=2), 3)]
    probs, refs = [], []
    for k, (g, tile) in enumerate(specs):
        plan = pnp.Plan(g)
        plan.set_launch_shapes(tile=tile)
        x = np.stack([f32(synth.ellipse_phantom(g.n, 90 + 5 * k + i, (4, 7))) for i in range(g.batch)])
        b = f32(np.stack([oracle.project(g, 1, xi) for xi in x]))
        stages = [synth.Stage(2, 3, 1), synth.Stage(1, 3, 2)]
        seq = synth.schedule_sequence(stages, k)
        eta = [0.8 / oracle.power_iter(g, s.factor, 60, 1e-7)[0] for s in stages]
        probs.append(dict(plan=plan, stages=stages, eta=eta, seq=seq, b=dev(b),
                          x=torch.zeros(g.batch, g.n, g.n, device="cuda"), xtrue=dev(x)))
        refs.append((g, stages, eta, seq, b, x))
    logs = pnp.run_many(probs)
    for pr, (g, stages, eta, seq, b, x), log in zip(probs, refs, logs):
        got = host(pr["x"])
        for i in range(g.batch):
            xr, lr = oracle.pnp_run(g, stages, eta, seq, b[i], None, xt=x[i])
            assert rel(got[i], xr) < TOL_RECON
            assert np.abs(log[:, i] - lr).max() < 1e-3


@pytest.mark.parametrize("n,batch,tv_iters", [(200, 2, 20), (130, 3, 13), (37, 1, 20)])
def test_strip_heights_agree_bitwise(n, batch, tv_iters):
    """The strips compute every kept value with the arithmetic of a global FGP
    iteration, so the three CTA heights (64, 96 and 128 rows: different tilings and
    halos) give the same bits, and all the oracle's denoiser output within 1e-5."""
    import torch
    g = synth.make_geometry(n, 30, int(1.5 * n), batch=batch)
    rng = np.random.default_rng(n)
    z = f32(rng.random((batch, n, n)))
    outs = []
    for tile in (2, 3, 4):
        plan = pnp.Plan(g)
        plan.set_launch_shapes(tile=tile)
        d_x = dev(z)
        # a zero-step run: the gradient term vanishes and x = D(z) (alpha 1, no momentum)
        plan.run([synth.Stage(1, 1, 1)], [0.0], None, dev(np.zeros((batch, 30, g.n_det))), d_x,
                 alpha=1.0, lam=0.05, tv_iters=tv_iters, momentum=False)
        outs.append(host(d_x))
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
    for i in range(batch):
        ref = oracle.fgp(z[i], 0.05, tv_iters)
        assert rel(outs[0][i], ref) < 1e-5, rel(outs[0][i], ref)
