"""GPU-vs-oracle parity of every step of the hot path, through the C ABI.

Tolerances (relative L2 = ||gpu - oracle|| / ||oracle||), from the FP32
arithmetic of the kernels against the FP64 oracle: 1e-5 for projections,
backprojections, gradients and the TV denoiser (sums of a few thousand FP32
terms of magnitude <= the result); 1e-4 for whole reconstructions, whose
errors accumulate over the iterations.  Inputs are identical on both sides:
the oracle receives the float32-rounded values the GPU receives.
"""
import math

import numpy as np
import pytest

import oracle
import paper_2203_07308_gb300 as pnp
from paper_2203_07308_gb300 import build, synth

pytestmark = pytest.mark.gpu

TOL = 1e-5
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
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def empty(*shape):
    import torch
    return torch.empty(*shape, dtype=torch.float32, device="cuda")


GEOMS = {
    "c1": synth.make_geometry(64, 90, 96, batch=2),
    # ragged: side not a multiple of the 16x16 block, odd bins, views not a multiple of P
    "ragged": synth.make_geometry(60, 37, 101, batch=3),
    # limited angle, one extra-wide detector (edge rays miss the image entirely)
    "limited": synth.Geometry(n=48, n_views=30, n_det=140, batch=1, dso=96.0, ddo=80.0,
                              det_pitch=2.3, angle0=0.3, angle_span=math.pi),
    "oneview": synth.make_geometry(32, 1, 48, batch=1),
    # steps other than half a pixel (generic sample-window paths)
    "step03": synth.make_geometry(40, 20, 64, batch=2, step=0.3),
    "step08": synth.make_geometry(36, 24, 60, batch=1, step=0.8),
}


def phantoms(g, seed=0):
    return np.stack([f32(synth.ellipse_phantom(g.n, 100 + seed + i, (6, 9))) for i in range(g.batch)])


@pytest.mark.parametrize("name", list(GEOMS))
@pytest.mark.parametrize("s", [1, 2, 4])
def test_forward_parity(name, s):
    g = GEOMS[name]
    if g.n % s or g.n // s < 4:
        pytest.skip("level not available")
    plan = pnp.Plan(g)
    x = phantoms(g)
    xs = np.stack([f32(oracle.pool(xi, s)) for xi in x])
    rng = np.random.default_rng(1)
    b = f32(rng.standard_normal((g.batch, g.n_views, g.n_det)) * 10)
    for P in sorted({1, min(4, g.n_views), g.n_views}):
        for p in sorted({0, P - 1}):
            nsub = pnp.subset_views(g, p, P)
            out = empty(g.batch, nsub, g.n_det)
            plan.project(s, dev(xs), out, None, p, P)
            got = host(out)
            ref = np.stack([oracle.project(g, s, xs[i], None, p, P) for i in range(g.batch)])
            assert rel(got, ref) < TOL, (name, s, P, p, rel(got, ref))
            plan.project(s, dev(xs), out, dev(b), p, P)
            got = host(out)
            ref = np.stack([oracle.project(g, s, xs[i], b[i], p, P) for i in range(g.batch)])
            assert rel(got, ref) < TOL


@pytest.mark.parametrize("name", list(GEOMS))
@pytest.mark.parametrize("s", [1, 2, 4])
def test_backward_parity_and_adjoint(name, s):
    g = GEOMS[name]
    if g.n % s or g.n // s < 4:
        pytest.skip("level not available")
    plan = pnp.Plan(g)
    ns = g.n // s
    rng = np.random.default_rng(2)
    for P in sorted({1, min(3, g.n_views)}):
        p = P - 1
        nsub = pnp.subset_views(g, p, P)
        y = f32(rng.standard_normal((g.batch, nsub, g.n_det)))
        out = empty(g.batch, ns, ns)
        plan.backproject(s, dev(y), out, p, P)
        got = host(out)
        ref = np.stack([oracle.backproject(g, s, y[i], p, P) for i in range(g.batch)])
        assert rel(got, ref) < TOL, (name, s, P, rel(got, ref))
        # FP32 adjoint identity on the GPU pair
        x = f32(rng.random((g.batch, ns, ns)))
        ax = empty(g.batch, nsub, g.n_det)
        plan.project(s, dev(x), ax, None, p, P)
        lhs = float(np.vdot(host(ax), y))
        rhs = float(np.vdot(x, got))
        assert abs(lhs - rhs) <= 1e-5 * (np.abs(host(ax)).sum() * np.abs(y).max())


def test_backprojection_is_bitwise_repeatable():
    g = GEOMS["c1"]
    plan = pnp.Plan(g)
    y = dev(np.random.default_rng(3).standard_normal((g.batch, g.n_views, g.n_det)))
    a, b = empty(g.batch, g.n, g.n), empty(g.batch, g.n, g.n)
    plan.backproject(1, y, a)
    plan.backproject(1, y, b)
    assert np.array_equal(host(a), host(b))


@pytest.mark.parametrize("s", [2, 4])
def test_sketch_and_upsample(s):
    g = GEOMS["c1"]
    x = f32(np.random.default_rng(4).random((g.batch, g.n, g.n)))
    c = empty(g.batch, g.n // s, g.n // s)
    pnp.sketch(g, s, dev(x), c)
    ref = np.stack([oracle.pool(xi, s) for xi in x])
    assert rel(host(c), ref) < 1e-7
    f = empty(g.batch, g.n, g.n)
    pnp.upsample(g, s, c, f)
    ref2 = np.stack([oracle.unpool(ci, s) for ci in host(c)])
    assert rel(host(f), ref2) < 1e-7


@pytest.mark.parametrize("name", ["c1", "ragged"])
@pytest.mark.parametrize("s,P", [(1, 1), (2, 1), (2, 5), (4, 3), (1, 8)])
def test_gradient_parity(name, s, P):
    g = GEOMS[name]
    if g.n % s or g.n // s < 4:
        pytest.skip("level not available")
    plan = pnp.Plan(g)
    x = phantoms(g, 5)
    rng = np.random.default_rng(6)
    b = f32(np.stack([oracle.project(g, 1, xi) for xi in x]) + rng.standard_normal((g.batch, g.n_views, g.n_det)))
    y = f32(rng.random((g.batch, g.n, g.n)))
    out = empty(g.batch, g.n, g.n)
    for p in sorted({0, P - 1}):
        plan.sketch_grad(s, dev(y), dev(b), out, p, P)
        ref = np.stack([oracle.grad(g, s, y[i], b[i], p, P) for i in range(g.batch)])
        assert rel(host(out), ref) < TOL, (name, s, P, p, rel(host(out), ref))
    if s == 1 and P == 1:
        plan.full_grad(dev(y), dev(b), out)
        assert rel(host(out), ref) < TOL


# one cluster per image with the state in registers (side a multiple of 32 and
# of the cluster size): 64, 96, 128, 256; with the state in shared memory: 37,
# 16, 200; several launches (state larger than one cluster): 512
@pytest.mark.parametrize("n,batch,lam,iters", [(64, 2, 0.02, 20), (96, 1, 0.04, 20), (128, 1, 0.05, 7),
                                               (256, 2, 0.02, 20), (37, 1, 0.1, 20), (16, 3, 0.3, 50),
                                               (200, 1, 0.02, 20), (512, 2, 0.02, 6)])
def test_tv_denoise_parity(n, batch, lam, iters):
    import torch
    rng = np.random.default_rng(n)
    z = f32(np.stack([synth.ellipse_phantom(n, 7 + i, (5, 5)) for i in range(batch)]) +
            0.1 * rng.standard_normal((batch, n, n)))
    ws = torch.empty(pnp.tv_workspace_size(n, batch), dtype=torch.uint8, device="cuda")
    out = empty(batch, n, n)
    pnp.tv_denoise(dev(z), out, n, batch, lam, iters, ws)
    ref = np.stack([oracle.fgp(z[i], lam, iters) for i in range(batch)])
    assert rel(host(out), ref) < TOL, rel(host(out), ref)
    pnp.tv_denoise(dev(z), out, n, batch, lam, 0, ws)
    assert np.array_equal(host(out), z)


@pytest.mark.parametrize("s", [1, 2])
def test_power_iteration_parity(s):
    g = synth.make_geometry(64, 90, 96)
    plan = pnp.Plan(g)
    L, it = plan.power_iter(s, 200, 1e-9)
    Lref, _ = oracle.power_iter(g, s, 200, 1e-9)
    assert abs(L - Lref) < 1e-5 * Lref, (L, Lref, it)


def test_objective_and_sample_count():
    g = GEOMS["c1"]
    plan = pnp.Plan(g)
    x = phantoms(g, 9)
    rng = np.random.default_rng(10)
    b = f32(np.stack([oracle.project(g, 1, xi) for xi in x]) + rng.standard_normal((g.batch, g.n_views, g.n_det)))
    xt = f32(x + 0.05 * rng.standard_normal(x.shape))
    out = plan.objective(dev(x), dev(b), dev(xt))
    for i in range(g.batch):
        f, tv = oracle.objective(g, x[i], b[i])
        assert abs(out[i, 0] - f) < 1e-5 * f
        assert abs(out[i, 1] - tv) < 1e-9 * tv
        assert abs(out[i, 2] - oracle.psnr(x[i], xt[i])) < 1e-9
    for s, P, p in [(1, 1, 0), (2, 1, 0), (1, 8, 3), (4, 5, 4)]:
        assert plan.sample_count(s, p, P) == oracle.sample_count(g, s, p, P)


def _run_both(g, stages, lam=0.02, tv_iters=20, momentum=True, alpha=1.0, seed=0):
    x = phantoms(g, 20 + seed)
    rng = np.random.default_rng(30 + seed)
    b = f32(np.stack([oracle.project(g, 1, xi) for xi in x]) +
            0.5 * rng.standard_normal((g.batch, g.n_views, g.n_det)))
    eta = [1.0 / oracle.power_iter(g, st.factor, 100, 1e-7)[0] for st in stages]
    seq = synth.schedule_sequence(stages, 7)
    plan = pnp.Plan(g)
    xg = dev(np.zeros((g.batch, g.n, g.n)))
    log = plan.run(stages, eta, seq, dev(b), xg, alpha=alpha, lam=lam, tv_iters=tv_iters,
                   momentum=momentum, xtrue=dev(x))
    got = host(xg)
    refs, logs = [], []
    for i in range(g.batch):
        xr, lr = oracle.pnp_run(g, stages, eta, seq, b[i], None, alpha=alpha, lam=lam,
                                tv_iters=tv_iters, momentum=momentum, xt=x[i])
        refs.append(xr)
        logs.append(lr)
    return got, np.stack(refs), log, np.stack(logs, axis=1)


def test_pnp_run_pgd_parity():
    """30 PnP-PGD iterations, full gradient (the 64x64 / 90 x 96 workload)."""
    g = synth.make_geometry(64, 90, 96, batch=1)
    got, ref, log, lref = _run_both(g, [synth.Stage(1, 30, 1)], momentum=False)
    assert rel(got, ref) < TOL_RECON, rel(got, ref)
    assert np.abs(log - lref).max() < 1e-3


def test_pnp_run_multistage_parity():
    """Three stages (4x, 2x, full) with angle subsets, FISTA momentum, alpha < 1, batch 2."""
    g = synth.make_geometry(64, 60, 96, batch=2)
    stages = [synth.Stage(4, 6, 3), synth.Stage(2, 6, 4), synth.Stage(1, 8, 5)]
    got, ref, log, lref = _run_both(g, stages, alpha=0.8, seed=1)
    assert rel(got, ref) < TOL_RECON, rel(got, ref)
    assert np.abs(log - lref).max() < 1e-3


def test_pnp_run_is_bitwise_repeatable():
    g = synth.make_geometry(64, 90, 96, batch=1)
    plan = pnp.Plan(g)
    stages = [synth.Stage(2, 4, 3), synth.Stage(1, 4, 3)]
    b = dev(np.random.default_rng(1).random((1, 90, 96)) * 30)
    seq = synth.schedule_sequence(stages, 3)
    outs = []
    for _ in range(2):
        x = dev(np.zeros((1, 64, 64)))
        plan.run(stages, [1e-4, 1e-4], seq, b, x)
        outs.append(host(x))
    assert np.array_equal(outs[0], outs[1])


# ------------------------------------------------------------ full-size workloads
def test_full_size_256_sampled_views():
    """The 256x256 / 360 views x 512 bins workload at full size: every kernel at
    the launch shape the benchmark uses; forward checked on sampled views (one
    view per oracle call), backprojection and gradient on the whole image."""
    wl = synth.workloads()["c2_256"]
    g = wl.geom
    plan = pnp.Plan(g)
    x = f32(synth.phantom_batch(wl))
    for s in (1, 2):
        xs = np.stack([f32(oracle.pool(xi, s)) for xi in x])
        out = empty(1, g.n_views, g.n_det)
        plan.project(s, dev(xs), out)
        got = host(out)[0]
        for v in (0, 47, 180, 359):
            ref = oracle.project(g, s, xs[0], None, v, g.n_views)[0]
            assert rel(got[v], ref) < TOL, (s, v, rel(got[v], ref))
    rng = np.random.default_rng(11)
    b = f32(rng.standard_normal((1, g.n_views, g.n_det)) * 20)
    y = f32(rng.random((1, g.n, g.n)))
    out = empty(1, g.n, g.n)
    plan.sketch_grad(2, dev(y), dev(b), out, 5, 8)
    ref = oracle.grad(g, 2, y[0], b[0], 5, 8)
    assert rel(host(out)[0], ref) < TOL


def test_full_size_512_batch16_sampled():
    """16 x 512x512 / 720 views x 768 bins: the batched launch at full size;
    two instances checked against the oracle on sampled views."""
    wl = synth.workloads()["c3_512x16"]
    g = wl.geom
    plan = pnp.Plan(g)
    x = f32(synth.phantom_batch(wl))
    out = empty(g.batch, g.n_views, g.n_det)
    plan.project(1, dev(x), out)
    got = host(out)
    for i in (0, 15):
        for v in (3, 500):
            ref = oracle.project(g, 1, x[i], None, v, g.n_views)[0]
            assert rel(got[i, v], ref) < TOL
    # backprojection of one angle subset (60 of 720 views), all instances
    P, p = 12, 5
    nsub = pnp.subset_views(g, p, P)
    y = f32(np.random.default_rng(12).standard_normal((g.batch, nsub, g.n_det)))
    img = empty(g.batch, g.n, g.n)
    plan.backproject(1, dev(y), img, p, P)
    got = host(img)
    ref = oracle.backproject(g, 1, y[7], p, P)
    assert rel(got[7], ref) < TOL, rel(got[7], ref)


# ------------------------------------------------------------ host-side errors on a GPU
def test_workspace_state_errors():
    import torch
    g = GEOMS["c1"]
    ws = torch.empty(pnp.workspace_size(g), dtype=torch.uint8, device="cuda")
    x = dev(np.zeros((g.batch, g.n, g.n)))
    out = empty(g.batch, g.n_views, g.n_det)
    with pytest.raises(pnp.PnpError) as e:
        pnp.project(g, 1, x, out, ws=ws)
    assert e.value.code == 5
    pnp.setup(g, ws)
    pnp.project(g, 1, x, out, ws=ws)
    g2 = synth.make_geometry(64, 91, 96, batch=2)
    with pytest.raises(pnp.PnpError) as e:
        pnp.project(g2, 1, x, empty(2, 91, 96), ws=ws)
    assert e.value.code == 5
