"""SVRG and SAGA subset estimates (Sec. 2 names them as replacements for the
vanilla minibatch gradient of Option 2) on the GPU: Algorithm 1 with
variance-reduced stages against the FP64 oracle, the estimator buffer's
state errors, and checkpoint/resume through the buffer."""
import numpy as np
import pytest

import oracle
import paper_2203_07308_gb300 as pnp
from paper_2203_07308_gb300 import _native, build, synth

pytestmark = pytest.mark.gpu
TOL_RECON = 1e-4
SVRG, SAGA = 1, 2


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


def problem(g, stages, seed):
    x = np.stack([f32(synth.ellipse_phantom(g.n, seed + i, (5, 8))) for i in range(g.batch)])
    rng = np.random.default_rng(seed)
    b = f32(np.stack([oracle.project(g, 1, xi) for xi in x]) + 0.3 * rng.standard_normal((g.batch, g.n_views, g.n_det)))
    eta = [0.5 / oracle.power_iter(g, s.factor, 60, 1e-7, kind=s.kind)[0] for s in stages]
    seq = synth.schedule_sequence(stages, seed)
    return x, b, eta, seq


@pytest.mark.parametrize("est", [SVRG, SAGA])
def test_vr_run_parity(est):
    """Three stages (4x bicubic, 2x pooled, full grid) with 3, 4 and 5 subsets,
    partial last epochs, FISTA momentum, alpha < 1, batch 2, TV denoiser."""
    import torch
    g = synth.make_geometry(64, 60, 96, batch=2)
    stages = [synth.Stage(4, 7, 3, kind=1, estimator=est), synth.Stage(2, 6, 4, estimator=est),
              synth.Stage(1, 7, 5, estimator=est)]
    x, b, eta, seq = problem(g, stages, 80 + est)
    plan = pnp.Plan(g)
    d_x = torch.zeros(2, 64, 64, device="cuda")
    log = plan.run(stages, eta, seq, dev(b), d_x, alpha=0.9, xtrue=dev(x))
    got = host(d_x)
    for i in range(2):
        xr, lr = oracle.pnp_run(g, stages, eta, seq, b[i], None, alpha=0.9, xt=x[i])
        assert rel(got[i], xr) < TOL_RECON, (i, rel(got[i], xr))
        assert np.abs(log[:, i] - lr).max() < 1e-3


def test_vr_and_minibatch_stages_mixed_with_another_class():
    """run_many: a class whose schedule mixes SAGA, vanilla and SVRG stages next
    to a vanilla class of another geometry; each against the oracle."""
    import torch
    ga = synth.make_geometry(64, 60, 96, batch=1)
    gb = synth.make_geometry(48, 40, 72, batch=2)
    sa = [synth.Stage(2, 5, 3, estimator=SAGA), synth.Stage(2, 3, 3), synth.Stage(1, 6, 4, estimator=SVRG)]
    sb = [synth.Stage(2, 4, 2), synth.Stage(1, 6, 3)]
    probs, refs = [], []
    for g, st, seed in ((ga, sa, 90), (gb, sb, 91)):
        x, b, eta, seq = problem(g, st, seed)
        d_x = torch.zeros(g.batch, g.n, g.n, device="cuda")
        probs.append(dict(plan=pnp.Plan(g), stages=st, eta=eta, seq=seq, b=dev(b), x=d_x))
        refs.append((g, st, eta, seq, b))
    pnp.run_many(probs)
    for pr, (g, st, eta, seq, b) in zip(probs, refs):
        got = host(pr["x"])
        for i in range(g.batch):
            xr, _ = oracle.pnp_run(g, st, eta, seq, b[i], None)
            assert rel(got[i], xr) < TOL_RECON, rel(got[i], xr)


def test_vr_buffer_state_errors():
    """A schedule with SVRG needs a registered estimator buffer of the size
    pnp_vr_buffer_size reports: none or a smaller one is PNP_ESTATE."""
    import torch
    g = synth.make_geometry(64, 60, 96, batch=1)
    stages = [synth.Stage(2, 3, 3, estimator=SVRG)]
    plan = pnp.Plan(g)
    b = torch.zeros(1, 60, 96, device="cuda")
    x = torch.zeros(1, 64, 64, device="cuda")
    seq = synth.schedule_sequence(stages, 1)
    with pytest.raises(pnp.PnpError) as e:
        _native.run(g, stages, [1e-4], seq, b, x, ws=plan.ws)
    assert e.value.code == _native.PNP_ESTATE
    need = pnp.vr_buffer_size(g, stages)
    plan.set_vr_buffer(torch.empty(need - 256, dtype=torch.uint8, device="cuda"))
    with pytest.raises(pnp.PnpError) as e:
        _native.run(g, stages, [1e-4], seq, b, x, ws=plan.ws)
    assert e.value.code == _native.PNP_ESTATE
    plan.set_vr_buffer(torch.empty(need, dtype=torch.uint8, device="cuda"))
    _native.run(g, stages, [1e-4], seq, b, x, ws=plan.ws)
    with pytest.raises(pnp.PnpError):
        _native.run(g, [synth.Stage(2, 3, 3, estimator=7)], [1e-4], seq, b, x, ws=plan.ws)


@pytest.mark.parametrize("est", [SVRG, SAGA])
def test_vr_checkpoint_resume_is_bitwise_identical(est):
    """Cut mid-epoch (iteration 5 of a stage with 3 subsets) and resume: the
    snapshot / table carried in the estimator buffer give the uninterrupted run
    bit for bit."""
    import torch
    g = synth.make_geometry(64, 60, 96, batch=2)
    stages = [synth.Stage(2, 8, 3, estimator=est), synth.Stage(1, 4, 4, estimator=est)]
    x, b, eta, seq = problem(g, stages, 95)
    plan = pnp.Plan(g)
    d_b = dev(b)
    full_x = torch.zeros(2, 64, 64, device="cuda")
    full_y = torch.zeros(2, 64, 64, device="cuda")
    pnp.run_many([dict(plan=plan, stages=stages, eta=eta, seq=seq, b=d_b, x=full_x, y=full_y)])
    k = 5
    cut = [synth.Stage(2, k, 3, estimator=est)]
    part_x = torch.zeros(2, 64, 64, device="cuda")
    part_y = torch.zeros(2, 64, 64, device="cuda")
    pnp.run_many([dict(plan=plan, stages=cut, eta=eta[:1], seq=seq[:k], b=d_b, x=part_x, y=part_y)])
    pnp.run_many([dict(plan=plan, stages=stages, eta=eta, seq=seq, b=d_b, x=part_x, y=part_y, start_iter=k)])
    assert np.array_equal(host(part_x), host(full_x))
    assert np.array_equal(host(part_y), host(full_y))
