"""Bicubic sketch S and upsampler U = S^T (Sec. 3: the paper's sketch and
upsampling operators are bicubic resizes) on the GPU against the FP64 oracle:
the resizes alone, the sketched gradient with and without angle subsets,
||A_s S||^2 by power iteration, and Algorithm 1 with bicubic stages."""
import numpy as np
import pytest

import oracle
import paper_2203_07308_gb300 as pnp
from paper_2203_07308_gb300 import build, synth

pytestmark = pytest.mark.gpu
TOL = 1e-5
TOL_RECON = 1e-4
BICUBIC = 1


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


def empty(*shape):
    import torch
    return torch.full(shape, float("nan"), device="cuda")


@pytest.mark.parametrize("n,s", [(64, 2), (64, 4), (96, 8), (40, 2), (256, 2)])
def test_bicubic_resizes(n, s):
    g = synth.make_geometry(n, 30, 48, batch=2)
    x = f32(np.random.default_rng(n + s).random((2, n, n)))
    c = empty(2, n // s, n // s)
    pnp.sketch(g, s, dev(x), c, kind=BICUBIC)
    ref = np.stack([oracle.bicubic_down(xi, s) for xi in x])
    assert rel(host(c), ref) < 1e-6, rel(host(c), ref)
    cf = f32(np.random.default_rng(s).standard_normal((2, n // s, n // s)))
    f = empty(2, n, n)
    pnp.upsample(g, s, dev(cf), f, kind=BICUBIC)
    ref2 = np.stack([oracle.bicubic_up(ci, s) for ci in cf])
    assert rel(host(f), ref2) < 1e-6, rel(host(f), ref2)


@pytest.mark.parametrize("s,P", [(2, 1), (2, 5), (4, 3), (8, 1)])
def test_bicubic_gradient_parity(s, P):
    g = synth.make_geometry(64, 60, 96, batch=2)
    plan = pnp.Plan(g)
    x = np.stack([f32(synth.ellipse_phantom(64, 40 + i, (5, 8))) for i in range(2)])
    rng = np.random.default_rng(41)
    b = f32(np.stack([oracle.project(g, 1, xi) for xi in x]) + rng.standard_normal((2, 60, 96)))
    y = f32(x + 0.1 * rng.standard_normal(x.shape))
    out = empty(2, 64, 64)
    for p in sorted({0, P - 1}):
        plan.sketch_grad(s, dev(y), dev(b), out, p, P, kind=BICUBIC)
        ref = np.stack([oracle.grad(g, s, y[i], b[i], p, P, kind=BICUBIC) for i in range(2)])
        assert rel(host(out), ref) < TOL, (p, rel(host(out), ref))


def test_bicubic_gradient_weighted():
    g = synth.make_geometry(64, 60, 96, batch=1)
    plan = pnp.Plan(g)
    x = f32(synth.ellipse_phantom(64, 50, (5, 8)))[None]
    bb, w = synth.poisson_transmission(oracle.project(g, 1, x[0]), 10 ** 4.5, 51)
    b, w = f32(bb)[None], f32(w)[None]
    plan.set_weights(dev(w))
    y = f32(np.random.default_rng(52).random((1, 64, 64)))
    out = empty(1, 64, 64)
    plan.sketch_grad(2, dev(y), dev(b), out, 1, 3, kind=BICUBIC)
    ref = oracle.grad(g, 2, y[0], b[0], 1, 3, w=w[0], kind=BICUBIC)
    assert rel(host(out)[0], ref) < TOL


@pytest.mark.parametrize("s", [2, 4])
def test_bicubic_power_iteration(s):
    g = synth.make_geometry(64, 90, 96)
    plan = pnp.Plan(g)
    L, it = plan.power_iter(s, 200, 1e-9, kind=BICUBIC)
    Lref, _ = oracle.power_iter(g, s, 200, 1e-9, kind=BICUBIC)
    assert abs(L - Lref) < 1e-5 * Lref, (L, Lref, it)
    Lpool, _ = oracle.power_iter(g, s, 200, 1e-9)
    assert abs(Lpool - Lref) > 1e-3 * Lref      # the two sketches are different operators


def test_pnp_run_bicubic_stages():
    """Algorithm 1 with bicubic sketched stages, angle subsets and a pooled
    stage in between, batch 2, against the oracle's run image by image."""
    g = synth.make_geometry(64, 60, 96, batch=2)
    stages = [synth.Stage(4, 5, 3, kind=BICUBIC), synth.Stage(2, 5, 1, kind=0),
              synth.Stage(2, 5, 4, kind=BICUBIC), synth.Stage(1, 6, 2)]
    x = np.stack([f32(synth.ellipse_phantom(64, 60 + i, (5, 8))) for i in range(2)])
    rng = np.random.default_rng(61)
    b = f32(np.stack([oracle.project(g, 1, xi) for xi in x]) + 0.5 * rng.standard_normal((2, 60, 96)))
    eta = [1.0 / oracle.power_iter(g, st.factor, 100, 1e-7, kind=st.kind)[0] for st in stages]
    seq = synth.schedule_sequence(stages, 9)
    plan = pnp.Plan(g)
    xg = dev(np.zeros((2, 64, 64)))
    log = plan.run(stages, eta, seq, dev(b), xg, alpha=0.9, xtrue=dev(x))
    got = host(xg)
    for i in range(2):
        xr, lr = oracle.pnp_run(g, stages, eta, seq, b[i], None, alpha=0.9, xt=x[i])
        assert rel(got[i], xr) < TOL_RECON, (i, rel(got[i], xr))
        assert np.abs(log[:, i] - lr).max() < 1e-3


def test_bicubic_run_many_mixed_classes():
    """run_many with one bicubic-sketch class and one pooled class of another
    geometry in the same call, each against its own single-class run."""
    import torch
    ga = synth.make_geometry(64, 60, 96, batch=2)
    gb = synth.make_geometry(48, 40, 72, batch=1)
    sa = [synth.Stage(2, 4, 3, kind=BICUBIC), synth.Stage(1, 3, 1)]
    sb = [synth.Stage(2, 4, 1), synth.Stage(1, 3, 2)]
    rng = np.random.default_rng(70)
    ba = dev(rng.random((2, 60, 96)) * 20)
    bbv = dev(rng.random((1, 40, 72)) * 20)
    ea, eb = [2e-4, 1e-4], [3e-4, 1e-4]
    qa, qb = synth.schedule_sequence(sa, 1), synth.schedule_sequence(sb, 2)
    pa, pb = pnp.Plan(ga), pnp.Plan(gb)
    solo = []
    for plan, st, e, q, b, g in ((pa, sa, ea, qa, ba, ga), (pb, sb, eb, qb, bbv, gb)):
        x = torch.zeros(g.batch, g.n, g.n, device="cuda")
        plan.run(st, e, q, b, x)
        solo.append(host(x))
    xa = torch.zeros(2, 64, 64, device="cuda")
    xb = torch.zeros(1, 48, 48, device="cuda")
    pnp.run_many([dict(plan=pa, stages=sa, eta=ea, seq=qa, b=ba, x=xa),
                  dict(plan=pb, stages=sb, eta=eb, seq=qb, b=bbv, x=xb)])
    # launch shapes may differ between a single class and a mixed call
    assert rel(host(xa), solo[0]) < 1e-6, rel(host(xa), solo[0])
    assert rel(host(xb), solo[1]) < 1e-6, rel(host(xb), solo[1])
