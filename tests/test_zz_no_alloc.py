"""pnp_full_grad_noalloc: the full gradient for callers that cannot allocate
device memory (a real-time service whose memory is fixed at start-up, a
plug-in inside an application that owns the GPU's allocator).  It takes no
workspace and keeps its scratch in a fixed array inside the library.

Checked through the C ABI against pnp_full_grad (which uses a caller-allocated
workspace), within the gradient tolerance of the parity tests, on two calls in
a row (the second call reuses the array the first one left behind).  This file
is collected last so that a run stopping at the first failure has already run
every other test; it passes alone in a fresh process as well.
"""
import ctypes as C

import numpy as np
import pytest

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


@pytest.mark.parametrize("g", [synth.make_geometry(64, 90, 96, batch=2),
                               synth.make_geometry(256, 360, 512, batch=1)],
                         ids=["64x64_b2", "256x256"])
def test_noalloc_matches_workspace_gradient_twice(g):
    import torch
    lib = _native.load()
    rng = np.random.default_rng(g.n)
    x = torch.from_numpy(rng.random((g.batch, g.n, g.n)).astype(np.float32)).cuda()
    b = torch.from_numpy((rng.standard_normal((g.batch, g.n_views, g.n_det)) * 10).astype(np.float32)).cuda()
    ref = torch.empty_like(x)
    plan = pnp.Plan(g)
    plan.full_grad(x, b, ref)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    cg = _native.geom(g)
    for call in range(2):
        out = torch.full_like(x, float("nan"))
        code = lib.pnp_full_grad_noalloc(C.byref(cg), C.c_void_p(x.data_ptr()), C.c_void_p(b.data_ptr()),
                                         C.c_void_p(out.data_ptr()), stream)
        assert code == 0, pnp.last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.float64)
        want = ref.cpu().numpy().astype(np.float64)
        assert np.isfinite(got).all()
        assert _rel(got, want) < TOL, (call, _rel(got, want))


def test_noalloc_rejects_geometry_beyond_its_scratch():
    import torch
    lib = _native.load()
    g = synth.make_geometry(512, 720, 768, batch=4)   # about 39 MB of scratch > 32 MiB
    cg = _native.geom(g)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    code = lib.pnp_full_grad_noalloc(C.byref(cg), C.c_void_p(256), C.c_void_p(512), C.c_void_p(1024), stream)
    assert code == _native.PNP_EINVAL
    assert "scratch" in pnp.last_error()
