"""pnp_full_grad_noalloc: the full gradient for callers that cannot allocate
device memory (a real-time service whose memory is fixed at start-up, a
plug-in inside an application that owns the GPU's allocator).  It takes no
workspace and keeps its scratch in a fixed array inside the library.

Checked through the C ABI against pnp_full_grad (which uses a caller-allocated
workspace) and against the FP64 oracle's gradient, within the gradient
tolerance of the parity tests, on two calls in a row (the second call reuses the
array the first one left behind), and on a small geometry after a large one (so
stale bytes left past the small call's scratch would show).  This file
is collected last so that a run stopping at the first failure has already run
every other test; it passes alone in a fresh process as well.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
import paper_2203_07308_gb300 as pnp
from paper_2203_07308_gb300 import _native, build, synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    pnp.load()


def _inputs(g):
    import torch
    rng = np.random.default_rng(g.n)
    x = rng.random((g.batch, g.n, g.n)).astype(np.float32)
    b = (rng.standard_normal((g.batch, g.n_views, g.n_det)) * 10).astype(np.float32)
    return x, b, torch.from_numpy(x).cuda(), torch.from_numpy(b).cuda()


def _noalloc(g, x, b):
    import torch
    lib = _native.load()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    out = torch.full_like(x, float("nan"))
    code = lib.pnp_full_grad_noalloc(C.byref(_native.geom(g)), C.c_void_p(x.data_ptr()), C.c_void_p(b.data_ptr()),
                                     C.c_void_p(out.data_ptr()), stream)
    assert code == 0, pnp.last_error()
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


GEOMS = [synth.make_geometry(64, 90, 96, batch=2), synth.make_geometry(256, 360, 512, batch=1),
         synth.make_geometry(64, 90, 96, batch=2)]


@pytest.mark.parametrize("g", GEOMS, ids=["64x64_b2", "256x256", "64x64_b2_after_256x256"])
def test_noalloc_matches_workspace_gradient_twice(g):
    import torch
    x_h, b_h, x, b = _inputs(g)
    ref = torch.empty_like(x)
    plan = pnp.Plan(g)
    plan.full_grad(x, b, ref)
    torch.cuda.synchronize()
    want = ref.cpu().numpy().astype(np.float64)
    orc = oracle.grad(g, 1, x_h[0].astype(np.float64), b_h[0].astype(np.float64))
    for call in range(2):
        got = _noalloc(g, x, b)
        assert np.isfinite(got).all()
        assert _rel(got, want) < TOL, (call, _rel(got, want))
        assert _rel(got[0], orc) < TOL, (call, _rel(got[0], orc))


def test_noalloc_rejects_geometry_beyond_its_scratch():
    import torch
    lib = _native.load()
    g = synth.make_geometry(512, 720, 768, batch=4)   # about 39 MB of scratch > 32 MiB
    cg = _native.geom(g)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    code = lib.pnp_full_grad_noalloc(C.byref(cg), C.c_void_p(256), C.c_void_p(512), C.c_void_p(1024), stream)
    assert code == _native.PNP_EINVAL
    assert "scratch" in pnp.last_error()
