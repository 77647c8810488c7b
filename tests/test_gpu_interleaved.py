"""Batches of at least 8 images keep their coefficient images image-interleaved
(one 128-byte line holds a cell of 8 images) and are projected by the forward
kernel that computes each sample's position once for 8, 16 or 32 images.  Checked
against the FP64 oracle on batches that fill lane groups exactly (8), leave a
ragged group (9), need 32-image chunks (40) or more than one staging chunk of the
coefficient-image kernel (70), at every sketch level, on angle subsets, with the
residual and weights of the gradient path."""
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


@pytest.mark.parametrize("n,views,det,batch", [(32, 20, 48, 8), (40, 24, 60, 9), (24, 16, 40, 40), (16, 12, 30, 70)])
def test_interleaved_forward_parity(n, views, det, batch):
    import torch
    g = synth.make_geometry(n, views, det, batch=batch)
    plan = pnp.Plan(g)
    rng = np.random.default_rng(batch)
    x = f32(rng.random((batch, n, n)))
    b = f32(rng.standard_normal((batch, views, det)))
    check = sorted({0, 3, batch // 2, batch - 1})
    for s in (1, 2, 4):
        if n % s or n // s < 4 or g.dso < np.sqrt(2.0) * (0.5 * n + 5.5 * s):
            continue                      # level not available for this geometry
        ns = n // s
        v = f32(x[:, ::s, ::s][:, :ns, :ns])
        for P, p in ((1, 0), (5, 3)):
            nsub = pnp.subset_views(g, p, P)
            out = torch.empty(batch, nsub, det, device="cuda")
            plan.project(s, dev(v), out, dev(b), p, P)
            got = host(out)
            for i in check:
                ref = oracle.project(g, s, v[i], b[i], p, P)
                assert rel(got[i], ref) < TOL, (s, P, i, rel(got[i], ref))


def test_interleaved_gradient_weighted_parity():
    """The sketched gradient of a 12-image batch (interleaved coefficient image at
    the 2x level, the pooled prep kernel) with WLS weights against the oracle."""
    g = synth.make_geometry(48, 30, 72, batch=12)
    plan = pnp.Plan(g)
    rng = np.random.default_rng(12)
    y = f32(rng.random((12, 48, 48)))
    b = f32(rng.standard_normal((12, 30, 72)) * 4)
    w = f32(rng.uniform(0.5, 2.0, (12, 30, 72)))
    plan.set_weights(dev(w))
    import torch
    out = torch.empty(12, 48, 48, device="cuda")
    plan.sketch_grad(2, dev(y), dev(b), out, 2, 3)
    got = host(out)
    for i in (0, 7, 11):
        ref = oracle.grad(g, 2, y[i], b[i], 2, 3, w=w[i])
        assert rel(got[i], ref) < TOL, (i, rel(got[i], ref))


@pytest.mark.parametrize("back", [8, 1 << 8 | 16, 4 << 16 | 4, 8 << 16 | 1 << 8 | 8, 16 << 16 | 8, 1 << 9 | 16])
@pytest.mark.parametrize("batch", [12, 10])
def test_interleaved_residual_every_backprojector_shape(back, batch):
    """Inside the gradient path the residual of an interleaved batch is stored
    image-interleaved too; every backprojector form reads it (the batched gather
    with 16-byte loads when the batch is a multiple of 4, scalar loads otherwise):
    the sketched subset gradient against the oracle."""
    import torch
    g = synth.make_geometry(40, 24, 60, batch=batch)
    plan = pnp.Plan(g)
    plan.set_launch_shapes(back=(back,) * 4)
    rng = np.random.default_rng(batch)
    y = f32(rng.random((batch, 40, 40)))
    b = f32(rng.standard_normal((batch, 24, 60)) * 3)
    for s, p, P in ((1, 1, 3), (2, 0, 1)):
        out = torch.empty(batch, 40, 40, device="cuda")
        plan.sketch_grad(s, dev(y), dev(b), out, p, P)
        got = host(out)
        for i in (0, batch - 1):
            ref = oracle.grad(g, s, y[i], b[i], p, P)
            assert rel(got[i], ref) < TOL, (back, s, i, rel(got[i], ref))
