"""Degenerate and edge cases on the GPU against the FP64 oracle or exact
identities: empty schedules and stages, the smallest image, a one-bin
detector, a one-view subset per iteration, data the iterate already explains
(zero residual gives an exactly zero gradient), a detector wider than the
fan so that most rays miss the image, and an image pointer that is not
vector-aligned."""
import numpy as np
import pytest

import oracle
import paper_2203_07308_gb300 as pnp
from paper_2203_07308_gb300 import build, synth

pytestmark = pytest.mark.gpu
TOL = 1e-5


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


def test_empty_schedule_and_empty_stage():
    """A schedule of zero iterations leaves x_0 untouched; a zero-iteration stage
    between two others changes nothing."""
    g = synth.make_geometry(32, 20, 48, batch=2)
    plan = pnp.Plan(g)
    rng = np.random.default_rng(1)
    x0 = f32(rng.random((2, 32, 32)))
    b = dev(rng.random((2, 20, 48)) * 10)
    x = dev(x0)
    plan.run([synth.Stage(2, 0, 1), synth.Stage(1, 0, 1)], [1e-3, 1e-3], [], b, x)
    assert np.array_equal(host(x), x0)
    a, c = dev(x0), dev(x0)
    seq = [1, 0, 2, 1]
    plan.run([synth.Stage(2, 2, 3), synth.Stage(1, 2, 3)], [1e-3, 1e-3], seq, b, a)
    plan.run([synth.Stage(2, 2, 3), synth.Stage(4, 0, 1), synth.Stage(1, 2, 3)], [1e-3, 5.0, 1e-3], seq, b, c)
    assert np.array_equal(host(a), host(c))


def test_smallest_image_and_one_bin_detector():
    import torch
    smallest = synth.Geometry(n=4, n_views=6, n_det=8, batch=1, dso=16.0, ddo=16.0,
                              det_pitch=synth.flat_detector_pitch(4, 8, 16.0, 16.0))
    one_bin = synth.Geometry(n=16, n_views=12, n_det=1, batch=2, dso=32.0, ddo=32.0, det_pitch=1.0)
    for g in (smallest, one_bin):
        plan = pnp.Plan(g)
        rng = np.random.default_rng(g.n)
        x = f32(rng.random((g.batch, g.n, g.n)))
        sino = torch.empty(g.batch, g.n_views, g.n_det, device="cuda")
        plan.project(1, dev(x), sino)
        ref = np.stack([oracle.project(g, 1, xi) for xi in x])
        assert rel(host(sino), ref) < TOL
        y = f32(rng.standard_normal((g.batch, g.n_views, g.n_det)))
        img = torch.empty(g.batch, g.n, g.n, device="cuda")
        plan.backproject(1, dev(y), img)
        ref = np.stack([oracle.backproject(g, 1, yi) for yi in y])
        assert rel(host(img), ref) < TOL


def test_one_view_per_subset():
    """P = n_views: every iteration uses a single view (c = n_views)."""
    g = synth.make_geometry(32, 12, 48, batch=1)
    plan = pnp.Plan(g)
    x = f32(synth.ellipse_phantom(32, 3, (3, 5)))[None]
    b = f32(oracle.project(g, 1, x[0]))[None]
    stages = [synth.Stage(1, 12, 12)]
    seq = synth.schedule_sequence(stages, 4)
    eta = [0.2 / oracle.power_iter(g, 1, 60, 1e-7)[0]]
    d_x = dev(np.zeros((1, 32, 32)))
    plan.run(stages, eta, seq, dev(b), d_x, momentum=False)
    xr, _ = oracle.pnp_run(g, stages, eta, seq, b[0], None, momentum=False)
    assert rel(host(d_x)[0], xr) < 1e-4


def test_zero_residual_gives_zero_gradient():
    """b = A x computed by the same forward projector: the residual, hence the
    gradient at every level and subset, is exactly zero."""
    import torch
    g = synth.make_geometry(48, 30, 64, batch=2)
    plan = pnp.Plan(g)
    plan.set_launch_shapes(lanes=(8, 8, 8, 8))      # the same summation order for every call
    x = dev(np.random.default_rng(5).random((2, 48, 48)))
    out = torch.empty(2, 48, 48, device="cuda")
    for s, P in ((1, 1), (2, 3), (4, 5)):
        ns = 48 // s
        # the data the sketched operator produces from the sketched iterate
        b = torch.zeros(2, g.n_views, g.n_det, device="cuda")
        for p in range(P):
            sub = torch.empty(2, pnp.subset_views(g, p, P), g.n_det, device="cuda")
            pool = torch.empty(2, ns, ns, device="cuda")
            pnp.sketch(g, s, x, pool) if s > 1 else pool.copy_(x)
            plan.project(s, pool, sub, None, p, P)
            b[:, p::P] = sub
        for p in range(P):
            plan.sketch_grad(s, x, b, out, p, P)
            assert float(out.abs().max()) == 0.0, (s, P, p)


def test_detector_wider_than_the_fan():
    """Most rays of a detector four times wider than the fan miss the image:
    their projections are exactly zero and the gradient still matches."""
    import torch
    g0 = synth.make_geometry(32, 16, 48, batch=1)
    g = synth.Geometry(n=32, n_views=16, n_det=192, batch=1, dso=g0.dso, ddo=g0.ddo,
                       det_pitch=g0.det_pitch, angle0=0.0, angle_span=g0.angle_span)
    plan = pnp.Plan(g)
    x = f32(synth.ellipse_phantom(32, 8, (3, 5)))[None]
    sino = torch.empty(1, 16, 192, device="cuda")
    plan.project(1, dev(x), sino)
    got = host(sino)[0]
    ref = oracle.project(g, 1, x[0])
    assert rel(got, ref) < TOL
    assert np.count_nonzero(ref == 0.0) > 16 * 100 and np.array_equal(got[ref == 0.0], ref[ref == 0.0])
    b = f32(ref + np.random.default_rng(9).standard_normal(ref.shape))[None]
    out = torch.empty(1, 32, 32, device="cuda")
    plan.full_grad(dev(x), dev(b), out)
    assert rel(host(out)[0], oracle.grad(g, 1, x[0], b[0])) < TOL


@pytest.mark.parametrize("batch", [8, 2])
def test_unaligned_image_pointer(batch):
    """An image that starts 4 bytes past an aligned address (a tensor view at
    storage offset 1) pooled by the sketch: the coefficient-image kernels then
    read it with scalar loads instead of one vector load per fine row, and the
    sketched gradient has the same bits as for an aligned copy, at the 2x and 4x
    levels, image-interleaved (batch 8) and image-major (batch 2)."""
    import torch
    n = 32
    g = synth.make_geometry(n, 30, 48, batch=batch)
    plan = pnp.Plan(g)
    rng = np.random.default_rng(8 + batch)
    y0 = rng.random((batch, n, n))
    b = dev(rng.standard_normal((batch, 30, 48)))
    ya = dev(y0)
    big = torch.zeros(1 + batch * n * n, device="cuda")
    yu = big[1:].view(batch, n, n)
    yu.copy_(ya)
    assert yu.data_ptr() % 16 == 4 and ya.data_ptr() % 16 == 0
    for s in (2, 4):
        for p, P in ((0, 1), (2, 3)):
            out_a = torch.empty(batch, n, n, device="cuda")
            out_u = torch.empty(batch, n, n, device="cuda")
            plan.sketch_grad(s, ya, b, out_a, p, P)
            plan.sketch_grad(s, yu, b, out_u, p, P)
            assert np.array_equal(host(out_a), host(out_u)), (s, p, P)
