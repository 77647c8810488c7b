"""Differentiable form on the GPU (through the C ABI and torch.autograd):
FGP reverse sweep, one unrolled iteration and its VJP, and the gradient of an
unrolled multi-stage run w.r.t. the input image x0 and the TV weight lambda,
against the FP64 oracle's reverse mode and against central finite differences
(h = 1e-3) of the GPU forward map.

Tolerances: relative 1e-4 for reverse-mode quantities (FP32 sums through up to
20 FGP iterations and several PnP iterations), 2e-2 for the FP32 finite
differences (step 1e-3 on values of order 1)."""
import numpy as np
import pytest

import oracle
import paper_2203_07308_gb300 as pnp
from paper_2203_07308_gb300 import _native, build, synth

pytestmark = pytest.mark.gpu

TOL_VJP = 1e-4
# Full-size unroll (10 iterations): the reconstruction bound 1e-4.  Measured on
# GB300: 1.5e-6 and 1.3e-5 for dJ/dx0 of the two checked instances, 1.4e-7 for
# dJ/dlambda; 1.0e-6, 1.5e-6 and 1.8e-5 at 5, 10 and 20 unrolled iterations
# (test_differentiable_error_growth_with_unrolled_iterations bounds the growth
# by 2 T x 1e-5: each of the T forward and T reverse gradient evaluations
# carries at most the single-gradient bound, and I - eta A^T A is
# non-expansive, so the errors add).
TOL_VJP_FULL = 1e-4


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
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("n,batch,lam,iters", [(32, 2, 0.05, 20), (45, 1, 0.1, 9)])
def test_tv_vjp_parity(n, batch, lam, iters):
    import torch
    rng = np.random.default_rng(n)
    z = f32(rng.random((batch, n, n)))
    xb = f32(rng.standard_normal((batch, n, n)))
    ws = torch.empty(_native.tv_vjp_workspace_size(n, batch, iters), dtype=torch.uint8, device="cuda")
    zb = torch.empty(batch, n, n, device="cuda")
    lb = _native.tv_vjp(dev(z), dev(xb), zb, n, batch, lam, iters, ws)
    got = host(zb)
    for i in range(batch):
        rz, rl = oracle.fgp_vjp(z[i], lam, iters, xb[i])
        assert rel(got[i], rz) < TOL_VJP, rel(got[i], rz)
        assert abs(lb[i] - rl) < TOL_VJP * max(1.0, abs(rl))


@pytest.mark.parametrize("s,P,p,alpha,amom", [(1, 1, 0, 1.0, 0.0), (2, 3, 2, 0.8, 0.3)])
def test_unrolled_step_and_vjp_parity(s, P, p, alpha, amom):
    import torch
    g = synth.make_geometry(48, 30, 64, batch=2)
    plan = pnp.Plan(g)
    rng = np.random.default_rng(s * 10 + p)
    b = f32(rng.standard_normal((2, g.n_views, g.n_det)) * 5)
    y = f32(rng.random((2, 48, 48)))
    xp = f32(rng.random((2, 48, 48)))
    xb = f32(rng.standard_normal((2, 48, 48)))
    yb = f32(rng.standard_normal((2, 48, 48)))
    eta, lam, it = 2e-4, 0.05, 20
    xo, yo = torch.empty(2, 48, 48, device="cuda"), torch.empty(2, 48, 48, device="cuda")
    _native.unrolled_step(g, s, p, P, eta, alpha, lam, it, amom, dev(y), dev(xp), dev(b), xo, yo, plan.ws)
    vws = torch.empty(_native.vjp_workspace_size(g, it), dtype=torch.uint8, device="cuda")
    ybi, xpb = torch.empty(2, 48, 48, device="cuda"), torch.empty(2, 48, 48, device="cuda")
    lb = _native.unrolled_step_vjp(g, s, p, P, eta, alpha, lam, it, amom, dev(y), dev(b), dev(xb), dev(yb),
                                   ybi, xpb, plan.ws, vws)
    for i in range(2):
        rx, ry = oracle.step(g, s, p, P, eta, alpha, lam, it, amom, y[i], xp[i], b[i])
        assert rel(host(xo)[i], rx) < 1e-5 and rel(host(yo)[i], ry) < 1e-5
        r_yb, r_xpb, r_lb = oracle.step_vjp(g, s, p, P, eta, alpha, lam, it, amom, y[i], b[i], xb[i], yb[i])
        assert rel(host(ybi)[i], r_yb) < TOL_VJP, rel(host(ybi)[i], r_yb)
        assert rel(host(xpb)[i], r_xpb) < 1e-6
        assert abs(lb[i] - r_lb) < TOL_VJP * max(1.0, abs(r_lb)), (lb[i], r_lb)
    # keeping z instead of recomputing it gives the same bits
    xo2, yo2, z = (torch.empty(2, 48, 48, device="cuda") for _ in range(3))
    _native.unrolled_step_save(g, s, p, P, eta, alpha, lam, it, amom, dev(y), dev(xp), dev(b), xo2, yo2, z,
                               plan.ws)
    assert np.array_equal(host(xo2), host(xo)) and np.array_equal(host(yo2), host(yo))
    ybi2, xpb2 = torch.empty(2, 48, 48, device="cuda"), torch.empty(2, 48, 48, device="cuda")
    lb2 = _native.unrolled_step_vjp_saved(g, s, p, P, eta, alpha, lam, it, amom, z, dev(xb), dev(yb), ybi2, xpb2,
                                          plan.ws, vws)
    assert np.array_equal(host(ybi2), host(ybi)) and np.array_equal(host(xpb2), host(xpb))
    assert np.array_equal(lb2, lb)


def _oracle_unrolled(g, stages, eta, seq, b, x0, xt, lam, alpha, tv_iters):
    ys, plan_ = [x0], []
    y, x = x0.copy(), x0.copy()
    i = 0
    for k, st in enumerate(stages):
        for _ in range(st.iters):
            i += 1
            p = int(seq[i - 1]) if st.n_subsets > 1 else 0
            a = (i - 1) / (i + 3)
            x, y = oracle.step(g, st.factor, p, st.n_subsets, eta[k], alpha, lam, tv_iters, a, y, x, b)
            ys.append(y)
            plan_.append((st.factor, p, st.n_subsets, eta[k], a))
    xb, yb, gl = x - xt, np.zeros_like(x), 0.0
    for t in range(len(plan_), 0, -1):
        s, p, P, e, a = plan_[t - 1]
        yb_in, xpb, lb = oracle.step_vjp(g, s, p, P, e, alpha, lam, tv_iters, a, ys[t - 1], b, xb, yb)
        gl += lb
        xb, yb = xpb, yb_in
    return 0.5 * np.sum((x - xt) ** 2), xb + yb, gl


@pytest.mark.parametrize("keep_z", [True, False])
def test_unrolled_autograd_matches_oracle_and_fd(keep_z):
    import torch
    from paper_2203_07308_gb300.autograd import unrolled_pnp
    g = synth.make_geometry(48, 36, 64, batch=2)
    plan = pnp.Plan(g)
    rng = np.random.default_rng(5)
    xt = np.stack([f32(synth.ellipse_phantom(48, 40 + i, (5, 7))) for i in range(2)])
    b = f32(np.stack([oracle.project(g, 1, x) for x in xt]) + 0.2 * rng.standard_normal((2, 36, 64)))
    stages = [synth.Stage(2, 2, 3), synth.Stage(1, 2, 2)]
    eta = [0.9 / oracle.power_iter(g, s.factor, 60, 1e-8)[0] for s in stages]
    seq = synth.schedule_sequence(stages, 11)
    x0 = f32(rng.random((2, 48, 48)) * 0.2)
    lam0, alpha, tvit = 0.03, 0.9, 12
    X0 = dev(x0).requires_grad_(True)
    lam = torch.tensor(lam0, dtype=torch.float64, requires_grad=True)
    xT = unrolled_pnp(plan, stages, eta, seq, dev(b), X0, lam, alpha=alpha, tv_iters=tvit, keep_z=keep_z)
    loss = 0.5 * ((xT - dev(xt)) ** 2).sum()
    loss.backward()
    gx = host(X0.grad)
    gl = float(lam.grad)
    ref_gl = 0.0
    for i in range(2):
        _, rgx, rgl = _oracle_unrolled(g, stages, eta, seq, b[i], x0[i], xt[i], lam0, alpha, tvit)
        assert rel(gx[i], rgx) < TOL_VJP, rel(gx[i], rgx)
        ref_gl += rgl
    assert abs(gl - ref_gl) < TOL_VJP * max(1.0, abs(ref_gl)), (gl, ref_gl)
    # central finite differences of the GPU forward map (float32), h = 1e-3
    def F(x0v, lv):
        with torch.no_grad():
            xx = unrolled_pnp(plan, stages, eta, seq, dev(b), dev(x0v), torch.tensor(lv, dtype=torch.float64),
                              alpha=alpha, tv_iters=tvit)
            return float(0.5 * ((xx.double() - dev(xt).double()) ** 2).sum())
    d = rng.standard_normal(x0.shape)
    d /= np.linalg.norm(d)
    h = 1e-3
    fdx = (F(x0 + h * d, lam0) - F(x0 - h * d, lam0)) / (2 * h)
    assert abs(fdx - np.vdot(gx, d)) < 2e-2 * max(1.0, abs(fdx))
    fdl = (F(x0, lam0 + h) - F(x0, lam0 - h)) / (2 * h)
    assert abs(fdl - gl) < 2e-2 * max(1.0, abs(fdl)), (fdl, gl)


_C4 = {}


def _c4_problem():
    """The differentiable workload (8 x 256x256, 360 views x 512 bins, 10 unrolled
    2x-sketched iterations) with data and step size from the oracle alone:
    b = A x_true + 1% noise (FP64 projection, rounded to FP32) and eta = 1/L of the
    oracle's power iteration."""
    if not _C4:
        wl = synth.workloads()["c4_256x8"]
        g = wl.geom
        xt = f32(synth.phantom_batch(wl))
        clean = np.stack([oracle.project(g, 1, xt[i]) for i in range(g.batch)])
        w = np.random.default_rng(4).standard_normal(clean.shape)
        b = f32(clean + 0.01 * np.abs(clean).max() * w)
        eta = [1.0 / oracle.power_iter(g, 2, 200, 1e-10)[0]]
        _C4.update(wl=wl, g=g, xt=xt, b=b, eta=eta)
    return _C4["wl"], _C4["g"], _C4["xt"], _C4["b"], _C4["eta"]


def _gpu_unrolled(plan, wl, stages, eta, seq, b, xt, x0, lam0, inst):
    """Loss 1/2 sum_{i in inst} ||x_T[i] - x_true[i]||^2 and its gradients w.r.t.
    x0 (all instances) and lambda through torch.autograd."""
    import torch
    from paper_2203_07308_gb300.autograd import unrolled_pnp
    X0 = dev(x0).requires_grad_(True)
    lam = torch.tensor(lam0, dtype=torch.float64, requires_grad=True)
    xT = unrolled_pnp(plan, stages, eta, seq, dev(b), X0, lam, alpha=wl.alpha, tv_iters=wl.tv_iters)
    sel = list(inst)
    loss = 0.5 * ((xT[sel] - dev(xt)[sel]) ** 2).sum()
    loss.backward()
    return float(loss), host(X0.grad), float(lam.grad)


def test_differentiable_workload_full_size():
    """8 x 256x256, 360 views x 512 bins, 10 unrolled 2x-sketched iterations, loss on
    instances 0 and 5: the gradient w.r.t. x0 of both and w.r.t. lambda (the sum of
    their two contributions) against the oracle's reverse mode; the other six
    instances run alongside and get a zero gradient."""
    wl, g, xt, b, eta = _c4_problem()
    plan = pnp.Plan(g)
    stages = wl.stages
    seq = synth.schedule_sequence(stages, 3)
    x0 = np.zeros((g.batch, g.n, g.n))
    _, gx, gl = _gpu_unrolled(plan, wl, stages, eta, seq, b, xt, x0, wl.tv_lambda, (0, 5))
    ref_gl = 0.0
    errs = {}
    for i in (0, 5):
        _, rgx, rgl = _oracle_unrolled(g, stages, eta, seq, b[i], x0[i], xt[i], wl.tv_lambda, wl.alpha,
                                       wl.tv_iters)
        errs[i] = rel(gx[i], rgx)
        ref_gl += rgl
    print("full-size unroll: relative error of dJ/dx0 per instance", errs, "dJ/dlambda", gl, ref_gl)
    for i, e in errs.items():
        assert e < TOL_VJP_FULL, (i, e)
    assert abs(gl - ref_gl) < TOL_VJP_FULL * abs(ref_gl), (gl, ref_gl)
    others = [i for i in range(g.batch) if i not in (0, 5)]
    assert not gx[others].any()


def test_differentiable_workload_full_size_finite_differences():
    """Central differences (h = 1e-3) of the GPU forward map at full size, against
    the autograd gradients: along a direction that mixes the gradient with a random
    unit vector (so the derivative is far above the FP32 noise of the loss, yet the
    check is not along the gradient alone), and along lambda."""
    import torch
    from paper_2203_07308_gb300.autograd import unrolled_pnp
    wl, g, xt, b, eta = _c4_problem()
    plan = pnp.Plan(g)
    stages = wl.stages
    seq = synth.schedule_sequence(stages, 3)
    x0 = f32(np.random.default_rng(8).random((g.batch, g.n, g.n)) * 0.1)
    inst = (0, 5)
    _, gx, gl = _gpu_unrolled(plan, wl, stages, eta, seq, b, xt, x0, wl.tv_lambda, inst)

    def F(x0v, lv):
        with torch.no_grad():
            xx = unrolled_pnp(plan, stages, eta, seq, dev(b), dev(x0v), torch.tensor(lv, dtype=torch.float64),
                              alpha=wl.alpha, tv_iters=wl.tv_iters)
            d_ = xx[list(inst)].double() - dev(xt)[list(inst)].double()
            return float(0.5 * (d_ ** 2).sum())
    u = np.random.default_rng(9).standard_normal(x0.shape)
    d = gx / np.linalg.norm(gx) + u / np.linalg.norm(u)
    d /= np.linalg.norm(d)
    h = 1e-3
    fdx = (F(x0 + h * d, wl.tv_lambda) - F(x0 - h * d, wl.tv_lambda)) / (2 * h)
    fdl = (F(x0, wl.tv_lambda + h) - F(x0, wl.tv_lambda - h)) / (2 * h)
    print("full-size finite differences: x0", fdx, np.vdot(gx, d), "lambda", fdl, gl)
    assert abs(fdx - np.vdot(gx, d)) < 2e-2 * abs(fdx)
    assert abs(fdl - gl) < 2e-2 * abs(fdl)


def test_differentiable_error_growth_with_unrolled_iterations():
    """The reverse-mode error of the full-size unroll against the oracle for T = 5,
    10 and 20 unrolled iterations (instance 0): each of the T forward and T reverse
    gradient evaluations carries at most the single-gradient bound, so the error
    stays below 2 T x 1e-5 and grows at most linearly in T."""
    wl, g, xt, b, eta = _c4_problem()
    plan = pnp.Plan(g)
    x0 = np.zeros((g.batch, g.n, g.n))
    errs = {}
    for T in (5, 10, 20):
        stages = [synth.Stage(2, T, 1)]
        seq = synth.schedule_sequence(stages, 3)
        _, gx, gl = _gpu_unrolled(plan, wl, stages, eta, seq, b, xt, x0, wl.tv_lambda, (0,))
        _, rgx, rgl = _oracle_unrolled(g, stages, eta, seq, b[0], x0[0], xt[0], wl.tv_lambda, wl.alpha,
                                       wl.tv_iters)
        errs[T] = (rel(gx[0], rgx), abs(gl - rgl) / abs(rgl))
    print("reverse-mode relative error by unrolled iterations (x0, lambda):", errs)
    for T, (ex, el) in errs.items():
        assert ex < 2 * T * 1e-5 and el < 2 * T * 1e-5, (T, ex, el)


@pytest.mark.parametrize("s,P,p", [(1, 1, 0), (2, 3, 1)])
def test_projector_autograd_functions(s, P, p):
    """Project / Backproject as autograd Functions: the autograd gradient of
    1/2 ||A_s v - b||^2 is the library's gradient and the oracle's A^T(A v - b);
    the two Functions are each other's adjoint through autograd."""
    import torch
    from paper_2203_07308_gb300.autograd import backproject, project
    g = synth.make_geometry(48, 30, 64, batch=2)
    plan = pnp.Plan(g)
    ns = 48 // s
    rng = np.random.default_rng(7 + s)
    v = f32(rng.random((2, ns, ns)))
    nsub = pnp.subset_views(g, p, P)
    b = f32(rng.standard_normal((2, nsub, g.n_det)) * 3)
    V = dev(v).requires_grad_(True)
    r = project(plan, V, s, p, P) - dev(b)
    (0.5 * (r ** 2).sum()).backward()
    got = host(V.grad)
    for i in range(2):
        ref = oracle.backproject(g, s, oracle.project(g, s, v[i], None, p, P) - b[i], p, P)
        assert rel(got[i], ref) < 1e-5, rel(got[i], ref)
    # Backproject's backward is the projector: d/dw <x, A^T w> = A x
    W = dev(b).requires_grad_(True)
    x = dev(rng.random((2, ns, ns)))
    (backproject(plan, W, s, p, P) * x).sum().backward()
    ax = torch.empty(2, nsub, g.n_det, device="cuda")
    plan.project(s, x, ax, None, p, P)
    assert np.array_equal(host(W.grad), host(ax))
