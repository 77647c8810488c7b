"""The paper's own set-ups on the GPU: weighted least squares for Poisson
transmission data (Sec. 3: b ~ Poisson(I0 exp(-A x)), then the log) and the
three fan-beam geometries of Sec. 3 (sparse-view, low-dose, limited-angle;
256x256, 228 bins), each against the FP64 oracle."""
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
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def poisson_problem(g, seed, i0=10 ** 4.5):
    x = np.stack([f32(synth.ellipse_phantom(g.n, seed + i, (6, 9))) for i in range(g.batch)])
    bs, ws = [], []
    for i in range(g.batch):
        b, w = synth.poisson_transmission(oracle.project(g, 1, x[i]), i0, seed + 100 + i)
        bs.append(b)
        ws.append(w)
    return x, f32(np.stack(bs)), f32(np.stack(ws))


@pytest.mark.parametrize("s,P", [(1, 1), (2, 4), (4, 3)])
def test_weighted_gradient_parity(s, P):
    import torch
    g = synth.make_geometry(64, 60, 96, batch=2)
    plan = pnp.Plan(g)
    x, b, w = poisson_problem(g, 3)
    plan.set_weights(dev(w))
    y = f32(np.random.default_rng(s).random((2, 64, 64)))
    out = torch.empty(2, 64, 64, device="cuda")
    for p in sorted({0, P - 1}):
        plan.sketch_grad(s, dev(y), dev(b), out, p, P)
        ref = np.stack([oracle.grad(g, s, y[i], b[i], p, P, w=w[i]) for i in range(2)])
        assert rel(host(out), ref) < TOL, rel(host(out), ref)
    plan.set_weights(None)
    plan.sketch_grad(s, dev(y), dev(b), out, 0, P)
    ref = np.stack([oracle.grad(g, s, y[i], b[i], 0, P) for i in range(2)])
    assert rel(host(out), ref) < TOL


def test_weighted_power_iteration_and_objective():
    g = synth.make_geometry(64, 60, 96, batch=1)
    plan = pnp.Plan(g)
    x, b, w = poisson_problem(g, 5)
    plan.set_weights(dev(w))
    L, _ = plan.power_iter(1, 200, 1e-9)
    Lref, _ = oracle.power_iter(g, 1, 200, 1e-9, w=w[0])
    assert abs(L - Lref) < 1e-5 * Lref
    out = plan.objective(dev(x), dev(b))
    f, tv = oracle.objective(g, x[0], b[0], w[0])
    assert abs(out[0, 0] - f) < 1e-5 * f


def test_weighted_pnp_run_parity():
    import torch
    g = synth.make_geometry(64, 60, 96, batch=2)
    plan = pnp.Plan(g)
    x, b, w = poisson_problem(g, 7)
    plan.set_weights(dev(w))
    stages = [synth.Stage(4, 3, 1), synth.Stage(2, 4, 1)]
    eta = [1.0 / oracle.power_iter(g, st.factor, 100, 1e-8, w=w[0])[0] for st in stages]
    d_x = torch.zeros(2, 64, 64, device="cuda")
    plan.run(stages, eta, None, dev(b), d_x)
    got = host(d_x)
    for i in range(2):
        rx, _ = oracle.pnp_run(g, stages, eta, [0] * 7, b[i], None, w=w[i])
        assert rel(got[i], rx) < TOL_RECON, rel(got[i], rx)


@pytest.mark.parametrize("name", ["sparse_view", "low_dose", "limited_angle"])
def test_paper_geometries(name):
    """A in R^{20520 x 65536} (90 views) or R^{82080 x 65536} (360 views), 228 bins."""
    import torch
    wl, i0 = synth.paper_workloads()[name]
    g = wl.geom
    assert g.n_views * g.n_det in (20520, 82080) and g.n * g.n == 65536
    plan = pnp.Plan(g)
    x = f32(synth.phantom_batch(wl, 1))
    sino = torch.empty(1, g.n_views, g.n_det, device="cuda")
    plan.project(1, dev(x), sino)
    got = host(sino)[0]
    for v in (0, g.n_views // 3, g.n_views - 1):
        ref = oracle.project(g, 1, x[0], None, v, g.n_views)[0]
        assert rel(got[v], ref) < TOL
    b, w = synth.poisson_transmission(oracle.project(g, 1, x[0]), i0, 21)
    b = f32(b)[None]
    w = f32(w)[None]
    plan.set_weights(dev(w))
    y = f32(np.random.default_rng(2).random((1, 256, 256)))
    gr = torch.empty(1, 256, 256, device="cuda")
    plan.sketch_grad(4, dev(y), dev(b), gr)
    ref = oracle.grad(g, 4, y[0], b[0], w=w[0])
    assert rel(host(gr)[0], ref) < TOL
