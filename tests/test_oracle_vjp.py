"""Pins of the oracle's reverse mode (the differentiable form) against central
finite differences of the oracle's own forward map in FP64: FGP, one iteration
of Algorithm 1, and a chain of iterations through the unrolled loss."""
import numpy as np
import pytest

import oracle
from paper_2203_07308_gb300 import synth


def fd(f, x, d, h):
    return (f(x + h * d) - f(x - h * d)) / (2 * h)


@pytest.mark.parametrize("lam,iters", [(0.1, 20), (0.03, 7), (0.5, 20)])
def test_fgp_vjp_matches_finite_differences(lam, iters):
    rng = np.random.default_rng(int(lam * 1000) + iters)
    z = rng.random((10, 10))
    xb = rng.standard_normal((10, 10))
    zb, lb = oracle.fgp_vjp(z, lam, iters, xb)
    J = lambda zz: np.vdot(xb, oracle.fgp(zz, lam, iters))
    for _ in range(3):
        d = rng.standard_normal(z.shape)
        assert abs(fd(J, z, d, 1e-6) - np.vdot(zb, d)) < 1e-6 * max(1.0, abs(np.vdot(zb, d)))
    Jl = lambda ll: np.vdot(xb, oracle.fgp(z, ll, iters))
    assert abs(fd(Jl, lam, 1.0, 1e-7) - lb) < 1e-5 * max(1.0, abs(lb))


def test_fgp_vjp_identity_cases():
    rng = np.random.default_rng(1)
    z = rng.random((6, 6))
    xb = rng.standard_normal((6, 6))
    zb, lb = oracle.fgp_vjp(z, 0.1, 0, xb)
    assert np.array_equal(zb, xb) and lb == 0.0


def _geom():
    return synth.make_geometry(16, 12, 24)


@pytest.mark.parametrize("s,P,p,alpha,amom", [(1, 1, 0, 1.0, 0.0), (2, 3, 1, 0.7, 0.4)])
def test_step_vjp_matches_finite_differences(s, P, p, alpha, amom):
    g = _geom()
    rng = np.random.default_rng(10 * s + p)
    b = rng.standard_normal((g.n_views, g.n_det)) * 4
    y = rng.random((16, 16))
    xp = rng.random((16, 16))
    eta, lam, it = 1e-3, 0.05, 15
    xb = rng.standard_normal((16, 16))
    yb = rng.standard_normal((16, 16))

    def J(yy, xx, ll):
        xo, yo = oracle.step(g, s, p, P, eta, alpha, ll, it, amom, yy, xx, b)
        return np.vdot(xb, xo) + np.vdot(yb, yo)

    ybi, xpb, lb = oracle.step_vjp(g, s, p, P, eta, alpha, lam, it, amom, y, b, xb, yb)
    d = rng.standard_normal(y.shape)
    assert abs(fd(lambda v: J(v, xp, lam), y, d, 1e-6) - np.vdot(ybi, d)) < 1e-6 * max(1, abs(np.vdot(ybi, d)))
    assert abs(fd(lambda v: J(y, v, lam), xp, d, 1e-6) - np.vdot(xpb, d)) < 1e-8 * max(1, abs(np.vdot(xpb, d)))
    assert abs(fd(lambda v: J(y, xp, v), lam, 1.0, 1e-7) - lb) < 1e-5 * max(1, abs(lb))


def unrolled_loss_and_grad(g, stages, eta, seq, b, x0, xt, lam, alpha=1.0, tv_iters=20, momentum=True):
    """Loss 1/2||x_T - xt||^2 of Algorithm 1 and its gradient w.r.t. (x0, lam),
    by chaining oracle.step_vjp backwards through the stored iterates."""
    ys, amoms, plan = [x0], [], []
    y, x = x0.copy(), x0.copy()
    i = 0
    for k, (s, N, P) in enumerate(stages):
        for _ in range(N):
            i += 1
            p = seq[i - 1] if P > 1 else 0
            a = (i - 1) / (i + 3) if momentum else 0.0
            x, y = oracle.step(g, s, p, P, eta[k], alpha, lam, tv_iters, a, y, x, b)
            ys.append(y)
            plan.append((s, p, P, eta[k], a))
    loss = 0.5 * np.sum((x - xt) ** 2)
    xb, yb = x - xt, np.zeros_like(x)
    lam_g = 0.0
    for t in range(len(plan), 0, -1):
        s, p, P, e, a = plan[t - 1]
        yb_in, xpb, lb = oracle.step_vjp(g, s, p, P, e, alpha, lam, tv_iters, a, ys[t - 1], b, xb, yb)
        lam_g += lb
        xb, yb = xpb, yb_in
    return loss, xb + yb, lam_g


def test_unrolled_chain_matches_finite_differences():
    g = _geom()
    rng = np.random.default_rng(7)
    xt = synth.ellipse_phantom(16, 3, (3, 3))
    b = np.asarray(oracle.project(g, 1, xt)) + 0.05 * rng.standard_normal((g.n_views, g.n_det))
    stages = [(2, 2, 3), (1, 2, 1)]
    eta = [0.5 / oracle.power_iter(g, 2, 50, 1e-9)[0], 0.5 / oracle.power_iter(g, 1, 50, 1e-9)[0]]
    seq = [2, 0, 0, 0]
    x0 = rng.random((16, 16)) * 0.3
    lam = 0.04
    loss, gx, gl = unrolled_loss_and_grad(g, stages, eta, seq, b, x0, xt, lam, alpha=0.9, tv_iters=10)
    f = lambda v: unrolled_loss_and_grad(g, stages, eta, seq, b, v, xt, lam, alpha=0.9, tv_iters=10)[0]
    d = rng.standard_normal(x0.shape)
    assert abs(fd(f, x0, d, 1e-6) - np.vdot(gx, d)) < 1e-6 * max(1.0, abs(np.vdot(gx, d)))
    fl = lambda v: unrolled_loss_and_grad(g, stages, eta, seq, b, x0, xt, v, alpha=0.9, tv_iters=10)[0]
    assert abs(fd(fl, lam, 1.0, 1e-7) - gl) < 1e-5 * max(1.0, abs(gl))
