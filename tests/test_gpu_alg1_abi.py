"""Algorithm 1 wholly behind the C ABI: step sizes eta_k = 1/L_k computed by the
library (Sec. 3: eta = O(1/L)) and the run without caller step sizes, checked
against the FP64 oracle's L and against runs given the same step sizes; the
unrolled form walking pnp_schedule; the seeded subset order drawn by the library
(pnp_subset_sequence) when no sequence is given."""
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


def test_step_sizes_match_the_oracle_and_the_power_iteration():
    """eta_k = 1/L_k per stage: the library's value equals 1/L of pnp_power_iter with
    the same settings exactly, and the FP64 oracle's 1/L within the gradient
    tolerance, for the pooled and the bicubic sketch; the cache is cleared by new
    weights."""
    g = synth.make_geometry(64, 90, 96, batch=2)
    plan = pnp.Plan(g)
    stages = [synth.Stage(4, 2, 3), synth.Stage(2, 2, 1, kind=1), synth.Stage(1, 3, 1)]
    eta = plan.step_sizes(stages)
    for st, e in zip(stages, eta):
        L, _ = plan.power_iter(st.factor, 100, 1e-6, kind=st.kind if st.factor > 1 else 0)
        assert e == 1.0 / L
        Lo, _ = oracle.power_iter(g, st.factor, 400, 1e-12, kind=st.kind if st.factor > 1 else 0)
        assert abs(e * Lo - 1.0) < TOL, (st, e * Lo)
    assert plan.step_sizes(stages) == eta                       # cached, same values
    w = np.random.default_rng(5).uniform(0.5, 2.0, (g.batch, g.n_views, g.n_det))
    plan.set_weights(dev(w))
    eta_w = plan.step_sizes(stages)
    Lw, _ = oracle.power_iter(g, 1, 400, 1e-12, w=np.asarray(w[0], np.float32).astype(np.float64))
    assert abs(eta_w[2] * Lw - 1.0) < TOL
    assert eta_w[2] != eta[2]


def test_run_without_step_sizes_equals_run_with_them():
    """pnp_run with h_eta = NULL gives the same bits as with h_eta = pnp_step_sizes,
    through pnp_run and pnp_run_many, with and without graph capture."""
    import torch
    g = synth.make_geometry(64, 90, 96, batch=2)
    plan = pnp.Plan(g)
    stages = [synth.Stage(2, 3, 3), synth.Stage(1, 4, 2)]
    seq = synth.schedule_sequence(stages, 11)
    x_true = np.stack([synth.ellipse_phantom(64, 300 + i, (6, 9)) for i in range(2)])
    b = torch.empty(2, g.n_views, g.n_det, device="cuda")
    plan.project(1, dev(x_true), b)
    outs = []
    for eta, graph in ((plan.step_sizes(stages), False), (None, False), (None, True)):
        x = torch.zeros(2, 64, 64, device="cuda")
        plan.run(stages, eta, seq, b, x, lam=0.02, tv_iters=20, momentum=True, graph=graph)
        outs.append(host(x))
    x = torch.zeros(2, 64, 64, device="cuda")
    pnp.run_many([dict(plan=plan, stages=stages, eta=None, seq=seq, b=b, x=x)], lam=0.02, tv_iters=20)
    outs.append(host(x))
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])


def test_run_without_step_sizes_matches_the_oracle_run():
    """The reconstruction with library step sizes against the oracle's run with its
    own FP64 step sizes (so the two sides share no input): within the
    reconstruction tolerance."""
    import torch
    g = synth.make_geometry(64, 90, 96)
    plan = pnp.Plan(g)
    stages = [synth.Stage(2, 4, 3), synth.Stage(1, 4, 1)]
    seq = synth.schedule_sequence(stages, 12)
    x_true = synth.ellipse_phantom(64, 77, (6, 9))
    b = oracle.project(g, 1, x_true)
    b = np.asarray(b, np.float32).astype(np.float64)
    x = torch.zeros(1, 64, 64, device="cuda")
    plan.run(stages, None, seq, dev(b[None]), x, lam=0.02, tv_iters=20, momentum=True)
    eta_o = [1.0 / oracle.power_iter(g, s.factor, 400, 1e-12)[0] for s in stages]
    xr, _ = oracle.pnp_run(g, stages, eta_o, seq, b, None, lam=0.02, tv_iters=20, momentum=True)
    got = host(x)[0]
    assert np.linalg.norm(got - xr) / np.linalg.norm(xr) < 1e-4


def test_unrolled_without_step_sizes_equals_with_them():
    """autograd.unrolled_pnp walks pnp_schedule; eta=None takes pnp_step_sizes: same
    x_T and gradients as the explicit step sizes."""
    import torch
    from paper_2203_07308_gb300.autograd import unrolled_pnp
    g = synth.make_geometry(48, 40, 64, batch=2)
    plan = pnp.Plan(g)
    stages = [synth.Stage(2, 2, 2), synth.Stage(1, 2, 1)]
    seq = synth.schedule_sequence(stages, 4)
    xt = dev(np.stack([synth.ellipse_phantom(48, 500 + i, (5, 7)) for i in range(2)]))
    b = torch.empty(2, g.n_views, g.n_det, device="cuda")
    plan.project(1, xt, b)
    res = []
    for eta in (plan.step_sizes(stages), None):
        x0 = torch.zeros(2, 48, 48, device="cuda", requires_grad=True)
        lam = torch.tensor(0.02, dtype=torch.float64, requires_grad=True)
        xT = unrolled_pnp(plan, stages, eta, seq, b, x0, lam, tv_iters=10)
        (0.5 * ((xT - xt) ** 2).sum()).backward()
        res.append((host(xT), host(x0.grad), float(lam.grad)))
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])
    assert res[0][2] == res[1][2]


def test_run_with_a_subset_seed_uses_the_seeded_order():
    """With no subset sequence the library draws the order from params.subset_seed
    (Sec. 2: the minibatch of each iteration is random): the same bits as a run
    given the oracle's order for that seed, through pnp_run (with and without
    graph capture), pnp_run_many and the unrolled form; within the
    reconstruction tolerance of the oracle's run on that order; another seed
    gives another reconstruction."""
    import torch
    from paper_2203_07308_gb300.autograd import unrolled_pnp
    g = synth.make_geometry(64, 90, 96, batch=2)
    plan = pnp.Plan(g)
    stages = [synth.Stage(2, 5, 3), synth.Stage(1, 6, 4)]
    seed = 2**63 + 5
    seq_o = oracle.subset_sequence(stages, seed)
    assert np.array_equal(pnp.subset_sequence(stages, seed), seq_o)
    x_true = np.stack([synth.ellipse_phantom(64, 320 + i, (6, 9)) for i in range(2)])
    b = oracle.project(g, 1, x_true[0]), oracle.project(g, 1, x_true[1])
    b = np.stack([np.asarray(v, np.float32) for v in b]).astype(np.float64)
    d_b = dev(b)
    eta = plan.step_sizes(stages)
    kw = dict(lam=0.02, tv_iters=20, momentum=True)
    x = torch.zeros(2, 64, 64, device="cuda")
    plan.run(stages, eta, seq_o, d_b, x, **kw)
    ref = host(x)
    for graph in (False, True):
        x = torch.zeros(2, 64, 64, device="cuda")
        plan.run(stages, eta, None, d_b, x, subset_seed=seed, graph=graph, **kw)
        assert np.array_equal(host(x), ref), graph
    x = torch.zeros(2, 64, 64, device="cuda")
    pnp.run_many([dict(plan=plan, stages=stages, eta=eta, seq=None, b=d_b, x=x)], subset_seed=seed, **kw)
    assert np.array_equal(host(x), ref)
    x = torch.zeros(2, 64, 64, device="cuda")
    plan.run(stages, eta, None, d_b, x, subset_seed=seed + 1, **kw)
    assert not np.array_equal(host(x), ref)
    xr, _ = oracle.pnp_run(g, stages, eta, seq_o, b[0], None, **kw)
    assert np.linalg.norm(ref[0] - xr) / np.linalg.norm(xr) < 1e-4
    x0 = torch.zeros(2, 64, 64, device="cuda")
    lam = torch.tensor(0.02, dtype=torch.float64)
    with torch.no_grad():
        xa = unrolled_pnp(plan, stages, eta, None, d_b, x0, lam, subset_seed=seed)
        xb = unrolled_pnp(plan, stages, eta, seq_o, d_b, x0, lam)
    assert np.array_equal(host(xa), host(xb))


def test_run_many_draws_each_class_order_from_its_own_stages():
    """pnp_run_many with two classes given no subset sequences: each class takes
    pnp_subset_sequence(its stages, params.subset_seed), so the call gives the
    same bits as the same call given the oracle's order for each class's stages;
    a class given a sequence keeps it.  (Several classes share one denoiser
    variant per launch, so the comparison is between calls on the same classes.)"""
    import torch
    ga = synth.make_geometry(64, 90, 96, batch=2)
    gb = synth.make_geometry(48, 60, 72, batch=1)
    pa, pb = pnp.Plan(ga), pnp.Plan(gb)
    sa = [synth.Stage(2, 4, 3), synth.Stage(1, 5, 6)]
    sb = [synth.Stage(1, 7, 5)]
    seed = 991
    kw = dict(lam=0.02, tv_iters=10, momentum=True)
    cls = []
    for g, plan, stages, pid in ((ga, pa, sa, 0), (gb, pb, sb, 1)):
        xt = np.stack([synth.ellipse_phantom(g.n, 40 + 7 * pid + i, (5, 8)) for i in range(g.batch)])
        b = torch.empty(g.batch, g.n_views, g.n_det, device="cuda")
        plan.project(1, dev(xt), b)
        cls.append(dict(plan=plan, stages=stages, eta=plan.step_sizes(stages), b=b, g=g))

    def call(seqs):
        xs = [torch.zeros(c["g"].batch, c["g"].n, c["g"].n, device="cuda") for c in cls]
        pnp.run_many([dict(plan=c["plan"], stages=c["stages"], eta=c["eta"], seq=q, b=c["b"], x=x)
                      for c, q, x in zip(cls, seqs, xs)], subset_seed=seed, **kw)
        return [host(x) for x in xs]

    ref = call([oracle.subset_sequence(sa, seed), oracle.subset_sequence(sb, seed)])
    got = call([None, None])
    assert all(np.array_equal(u, v) for u, v in zip(got, ref))
    own = synth.schedule_sequence(sb, 3)
    assert not np.array_equal(own, oracle.subset_sequence(sb, seed))
    ref2 = call([oracle.subset_sequence(sa, seed), own])
    got2 = call([None, own])
    assert all(np.array_equal(u, v) for u, v in zip(got2, ref2))
    assert not np.array_equal(got2[1], got[1])
