"""The stored gather table (pnp_set_gather_table, launch shapes with
PNP_BACK_TABLE): the gather's weights computed once per geometry and streamed
back from HBM.  Its sums are the bits of the gather with the same number of view
groups (the same weights, the same view and ray order, the same fixed-order
sum over the groups), which every case checks, on ragged sizes, rays that miss
the image, one view, sample steps other than half a pixel, every sketch level,
subsets, the three epilogues (raw, gradient, fused step) and whole runs of
Algorithm 1; plus the FP64 oracle, the size and argument checks, the fallback
without a table and a full-size 16 x 512^2 subset at every level."""
import ctypes as C
import math

import numpy as np
import pytest

import oracle
import paper_2203_07308_gb300 as pnp
from paper_2203_07308_gb300 import _native as N
from paper_2203_07308_gb300 import build, synth

pytestmark = pytest.mark.gpu
TOL = 1e-5

GEOMS = {
    "c1": synth.make_geometry(64, 90, 96, batch=2),
    "ragged5": synth.make_geometry(60, 37, 101, batch=5),
    "limited": synth.Geometry(n=48, n_views=30, n_det=140, batch=1, dso=96.0, ddo=80.0,
                              det_pitch=2.3, angle0=0.3, angle_span=math.pi),
    "oneview": synth.make_geometry(32, 1, 48, batch=1),
    "step03": synth.make_geometry(40, 20, 64, batch=4, step=0.3),
    "step08": synth.make_geometry(36, 24, 60, batch=9, step=0.8),
    "il16": synth.make_geometry(64, 36, 96, batch=16),
}


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
    return torch.full(shape, float("nan"), dtype=torch.float32, device="cuda")


def bc_of(batch):
    return 16 if batch >= 16 else 8 if batch >= 8 else 4


def batch_ok(batch):
    return batch >= 2                     # the batched gather (one image: the unbatched one)


def pair(g, G):
    """(the gather with G view groups, the table gather with G view groups)"""
    bc = bc_of(g.batch)
    ref_shape = (N.BACK_BATCH(bc) | G) if batch_ok(g.batch) else G
    ref = pnp.Plan(g)
    ref.set_launch_shapes(back=(ref_shape,) * 4)
    tab = pnp.Plan(g, gather_table=True)
    tab.set_launch_shapes(back=(N.BACK_TABLE | N.BACK_BATCH(bc) | G,) * 4)
    return ref, tab


def levels(g):
    return [s for s in (1, 2, 4) if g.n % s == 0 and g.n // s >= 4 and g.dso >= math.sqrt(2.0) * (0.5 * g.n + 5.5 * s)]


@pytest.mark.parametrize("G", [1, 4, 16])
@pytest.mark.parametrize("name", list(GEOMS))
def test_table_gather_bitwise_equals_the_gather(name, G):
    g = GEOMS[name]
    ref, tab = pair(g, G)
    rng = np.random.default_rng(G + len(name))
    for s in levels(g):
        ns = g.n // s
        for p, P in ((0, 1), (min(2, g.n_views - 1), min(3, g.n_views))):
            y = f32(rng.standard_normal((g.batch, pnp.subset_views(g, p, P), g.n_det)))
            o1, o2 = empty(g.batch, ns, ns), empty(g.batch, ns, ns)
            ref.backproject(s, dev(y), o1, p, P)
            tab.backproject(s, dev(y), o2, p, P)
            a, b = host(o1), host(o2)
            assert np.isfinite(b).all()
            assert np.array_equal(a, b), (s, p, P)
            if G == 4:
                want = oracle.backproject(g, s, y[-1], p, P)
                assert rel(b[-1], want) < TOL, (s, rel(b[-1], want))
    x = dev(rng.random((g.batch, g.n, g.n)))
    bb = dev(rng.standard_normal((g.batch, g.n_views, g.n_det)))
    for s in levels(g):
        o1, o2 = empty(g.batch, g.n, g.n), empty(g.batch, g.n, g.n)
        ref.sketch_grad(s, x, bb, o1, 0, min(2, g.n_views))
        tab.sketch_grad(s, x, bb, o2, 0, min(2, g.n_views))
        assert np.array_equal(host(o1), host(o2)), s


def test_table_runs_of_algorithm_1_bitwise_and_against_the_oracle():
    """Multi-stage runs with subsets, relaxation and momentum (the fused step
    epilogue): the table plan's iterates and PSNR logs equal the gather plan's."""
    g = synth.make_geometry(64, 60, 96, batch=3)
    ref, tab = pair(g, 8)
    x = np.stack([f32(synth.ellipse_phantom(64, 500 + i, (4, 7))) for i in range(3)])
    rng = np.random.default_rng(3)
    b = f32(np.stack([oracle.project(g, 1, xi) for xi in x]) + 0.2 * rng.standard_normal((3, 60, 96)))
    stages = [synth.Stage(2, 3, 4), synth.Stage(1, 4, 2)]
    seq = synth.schedule_sequence(stages, 4)
    eta = [0.8 / oracle.power_iter(g, s.factor, 60, 1e-7)[0] for s in stages]
    outs = []
    for plan in (ref, tab):
        d_x = dev(np.zeros((3, 64, 64)))
        log = plan.run(stages, eta, seq, dev(b), d_x, alpha=0.9, lam=0.03, tv_iters=8, xtrue=dev(x))
        outs.append((host(d_x), np.asarray(log)))
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1])
    for i in range(3):
        xr, _ = oracle.pnp_run(g, stages, eta, seq, b[i], None, alpha=0.9, lam=0.03, tv_iters=8, xt=x[i])
        assert rel(outs[1][0][i], xr) < 1e-4


def test_table_size_arguments_and_fallback():
    import torch
    g = synth.make_geometry(48, 40, 72, batch=2)
    plan = pnp.Plan(g)
    lib = N.load()
    need = plan.gather_table_size()
    groups = lambda ns: ((ns + 1) // 2) ** 2 // 32 + (1 if ((ns + 1) // 2) ** 2 % 32 else 0)
    assert need > 40 * groups(48) * 8                     # the full-grid level's header at least
    small = torch.empty(need - 256, dtype=torch.uint8, device="cuda")
    code = lib.pnp_set_gather_table(C.byref(plan.cg), C.c_void_p(small.data_ptr()), small.numel(),
                                    N._ws(plan.ws)[0], None)
    assert code == N.PNP_EINVAL and "too small" in pnp.last_error()
    buf = torch.empty(need + 512, dtype=torch.uint8, device="cuda")
    code = lib.pnp_set_gather_table(C.byref(plan.cg), C.c_void_p(buf.data_ptr() + 16), need,
                                    N._ws(plan.ws)[0], None)
    assert code == N.PNP_EINVAL and "aligned" in pnp.last_error()
    # the table shape without a registered table runs as the gather of the same groups
    plan.set_launch_shapes(back=(N.BACK_TABLE | N.BACK_BATCH(2) | 4,) * 4)
    rng = np.random.default_rng(48)
    y = f32(rng.standard_normal((2, 40, 72)))
    o1 = empty(2, 48, 48)
    plan.backproject(1, dev(y), o1)
    plan.set_gather_table()
    o2 = empty(2, 48, 48)
    plan.backproject(1, dev(y), o2)
    assert np.array_equal(host(o1), host(o2))
    want = oracle.backproject(g, 1, y[1])
    assert rel(host(o2)[1], want) < TOL
    # unregistering, and a fresh set-up, drop the table (the gather runs again)
    plan.set_gather_table(False)
    o3 = empty(2, 48, 48)
    plan.backproject(1, dev(y), o3)
    assert np.array_equal(host(o1), host(o3))
    with pytest.raises(pnp.PnpError):
        N._check(lib.pnp_gather_table_size(C.byref(plan.cg), N._ws(plan.ws)[0], None, None))


def test_autotune_with_a_table():
    """With a table registered the autotuner also times the table shapes; the
    gradient of whatever it picks matches the oracle."""
    g = synth.make_geometry(64, 90, 96, batch=4)
    plan = pnp.Plan(g, gather_table=True)
    stages = [synth.Stage(2, 4, 3), synth.Stage(1, 4, 3)]
    plan.autotune(stages, tv_iters=10)
    rng = np.random.default_rng(7)
    y = f32(rng.random((4, 64, 64)))
    b = f32(rng.standard_normal((4, 90, 96)))
    out = empty(4, 64, 64)
    plan.sketch_grad(1, dev(y), dev(b), out, 1, 3)
    ref = oracle.grad(g, 1, y[2], b[2], 1, 3)
    assert rel(host(out)[2], ref) < TOL


def test_full_size_512x16_table_bitwise_every_level():
    """16 x 512^2 / 720 x 768 (the benchmark's workload): one 60-view subset at
    each level, table gather against the batched gather with 8 view groups."""
    g = synth.workloads()["c3_512x16"].geom
    ref, tab = pair(g, 8)
    rng = np.random.default_rng(512)
    for s in (1, 2, 4):
        ns = g.n // s
        y = f32(rng.standard_normal((g.batch, pnp.subset_views(g, 5, 12), g.n_det)))
        o1, o2 = empty(g.batch, ns, ns), empty(g.batch, ns, ns)
        ref.backproject(s, dev(y), o1, 5, 12)
        tab.backproject(s, dev(y), o2, 5, 12)
        assert np.array_equal(host(o1), host(o2)), s
