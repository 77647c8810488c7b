"""Batched forms on the GPU: uneven classes of images (size, views, bins) in one
launch per phase (pnp_run_many), CUDA-graph replay, and autotuned launch
shapes, each against the FP64 oracle (relative L2 <= 1e-4 on reconstructions)."""
import numpy as np
import pytest

import oracle
import paper_2203_07308_gb300 as pnp
from paper_2203_07308_gb300 import build, synth

pytestmark = pytest.mark.gpu
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


def make_problem(g, stages, seed, lam=0.02):
    x = np.stack([f32(synth.ellipse_phantom(g.n, seed + i, (5, 8))) for i in range(g.batch)])
    rng = np.random.default_rng(seed)
    b = f32(np.stack([oracle.project(g, 1, xi) for xi in x]) +
            0.3 * rng.standard_normal((g.batch, g.n_views, g.n_det)))
    eta = [1.0 / oracle.power_iter(g, s.factor, 60, 1e-7)[0] for s in stages]
    seq = synth.schedule_sequence(stages, seed)
    return x, b, eta, seq


def oracle_runs(g, stages, eta, seq, b, x, lam, alpha=1.0, tv_iters=20):
    refs, logs = [], []
    for i in range(g.batch):
        xr, lr = oracle.pnp_run(g, stages, eta, seq, b[i], None, alpha=alpha, lam=lam, tv_iters=tv_iters,
                                momentum=True, xt=x[i])
        refs.append(xr)
        logs.append(lr)
    return np.stack(refs), np.stack(logs, axis=1)


def test_run_many_uneven_classes():
    """Three classes with different sizes, views, bins, batch sizes and schedule
    lengths in one call: every phase of every iteration is one launch."""
    import torch
    specs = [
        (synth.make_geometry(32, 20, 48, batch=3), [synth.Stage(2, 3, 4), synth.Stage(1, 4, 4)]),
        (synth.make_geometry(48, 36, 64, batch=1), [synth.Stage(4, 2, 3), synth.Stage(2, 2, 3), synth.Stage(1, 5, 2)]),
        (synth.make_geometry(64, 30, 96, batch=2), [synth.Stage(2, 5, 1)]),
    ]
    problems, refs = [], []
    launches0 = pnp.launch_count()
    for k, (g, stages) in enumerate(specs):
        x, b, eta, seq = make_problem(g, stages, 100 + 10 * k)
        plan = pnp.Plan(g)
        d_x = torch.zeros(g.batch, g.n, g.n, device="cuda")
        problems.append(dict(plan=plan, stages=stages, eta=eta, seq=seq, b=dev(b), x=d_x, xtrue=dev(x)))
        refs.append((g, stages, eta, seq, b, x))
    launches0 = pnp.launch_count()
    logs = pnp.run_many(problems, lam=0.02, tv_iters=20)
    launched = pnp.launch_count() - launches0
    max_iters = max(sum(s.iters for s in st) for _, st in specs)
    # per iteration: prep, forward, backprojection, two TV launches (10 FGP
    # iterations each), plus one PSNR reduction per class; one copy per class
    assert launched <= len(specs) + max_iters * (5 + len(specs)), launched
    for prob, (g, stages, eta, seq, b, x), log in zip(problems, refs, logs):
        rx, rl = oracle_runs(g, stages, eta, seq, b, x, 0.02)
        got = host(prob["x"])
        assert rel(got, rx) < TOL_RECON, rel(got, rx)
        assert np.abs(log - rl).max() < 1e-3


def test_run_many_more_classes_than_one_launch_holds():
    """Six classes (more than the four one launch covers): the phases run as one
    launch per group of four classes, with schedules of different lengths, a
    nine-image class (image-interleaved coefficient images) and the PSNR log;
    every class against the oracle."""
    import torch
    specs = [
        (synth.make_geometry(24, 16, 36, batch=2), [synth.Stage(2, 2, 3), synth.Stage(1, 2, 1)]),
        (synth.make_geometry(32, 20, 48, batch=1), [synth.Stage(1, 3, 2)]),
        (synth.make_geometry(28, 18, 40, batch=9), [synth.Stage(2, 3, 1)]),
        (synth.make_geometry(36, 24, 52, batch=1), [synth.Stage(4, 1, 1), synth.Stage(1, 4, 3)]),
        (synth.make_geometry(20, 12, 30, batch=3), [synth.Stage(1, 2, 1)]),
        (synth.make_geometry(40, 22, 56, batch=2), [synth.Stage(2, 2, 2), synth.Stage(1, 3, 2)]),
    ]
    problems, refs = [], []
    for k, (g, stages) in enumerate(specs):
        x, b, eta, seq = make_problem(g, stages, 300 + 10 * k)
        plan = pnp.Plan(g)
        d_x = torch.zeros(g.batch, g.n, g.n, device="cuda")
        problems.append(dict(plan=plan, stages=stages, eta=eta, seq=seq, b=dev(b), x=d_x, xtrue=dev(x)))
        refs.append((g, stages, eta, seq, b, x))
    logs = pnp.run_many(problems, lam=0.02, tv_iters=20)
    for prob, (g, stages, eta, seq, b, x), log in zip(problems, refs, logs):
        rx, rl = oracle_runs(g, stages, eta, seq, b, x, 0.02)
        got = host(prob["x"])
        assert rel(got, rx) < TOL_RECON, (g.n, rel(got, rx))
        assert np.abs(log - rl).max() < 1e-3


@pytest.mark.parametrize("back", [1 << 9 | 16, 1 << 8 | 8])
def test_run_many_takes_the_largest_class_shapes(back):
    """One launch per phase uses the tuned (here pinned) projector shapes of the
    class with the most level pixels: the fixed-point scatter or 4 x 4-block
    gather pinned on the 64^2 class runs every class's backprojection, and every
    class still matches the oracle."""
    import torch
    specs = [
        (synth.make_geometry(32, 20, 48, batch=3), [synth.Stage(2, 3, 4), synth.Stage(1, 4, 4)]),
        (synth.make_geometry(64, 30, 96, batch=2), [synth.Stage(2, 3, 1), synth.Stage(1, 3, 2)]),
    ]
    problems, refs = [], []
    for k, (g, stages) in enumerate(specs):
        x, b, eta, seq = make_problem(g, stages, 300 + 10 * k)
        plan = pnp.Plan(g)
        if g.n == 64:
            plan.set_launch_shapes(lanes=(4, 4, 0, 0), back=(back, back, 0, 0))
        d_x = torch.zeros(g.batch, g.n, g.n, device="cuda")
        problems.append(dict(plan=plan, stages=stages, eta=eta, seq=seq, b=dev(b), x=d_x, xtrue=dev(x)))
        refs.append((g, stages, eta, seq, b, x))
    logs = pnp.run_many(problems, lam=0.02, tv_iters=20)
    for prob, (g, stages, eta, seq, b, x), log in zip(problems, refs, logs):
        rx, rl = oracle_runs(g, stages, eta, seq, b, x, 0.02)
        got = host(prob["x"])
        assert rel(got, rx) < TOL_RECON, rel(got, rx)
        assert np.abs(log - rl).max() < 1e-3


def test_graph_replay_matches_direct_launches():
    import torch
    g = synth.make_geometry(64, 60, 96, batch=2)
    stages = [synth.Stage(2, 3, 5), synth.Stage(1, 3, 5)]
    x, b, eta, seq = make_problem(g, stages, 7)
    plan = pnp.Plan(g)
    outs = []
    for graph in (False, True, True):
        d_x = torch.zeros(g.batch, g.n, g.n, device="cuda")
        plan.run(stages, eta, seq, dev(b), d_x, graph=graph)
        outs.append(host(d_x))
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[1], outs[2])


def test_autotuned_shapes_keep_parity():
    import torch
    g = synth.make_geometry(64, 90, 96, batch=1)
    stages = [synth.Stage(2, 4, 3), synth.Stage(1, 4, 3)]
    x, b, eta, seq = make_problem(g, stages, 9)
    plan = pnp.Plan(g)
    plan.autotune(stages)
    d_x = torch.zeros(1, 64, 64, device="cuda")
    plan.run(stages, eta, seq, dev(b), d_x)
    rx, _ = oracle_runs(g, stages, eta, seq, b, x, 0.02)
    assert rel(host(d_x), rx) < TOL_RECON


def test_mixed_64_instances_full_size():
    """The 64-image uneven mix (128/180/256, 256/360/512, 512/720/768) at full
    size, 50 sketched iterations, one call; sampled 128x128 and 256x256 images
    against the oracle, every image finite and improved over x_0 = 0."""
    import torch
    classes = synth.mixed_classes()
    problems, meta = [], []
    for wl, ids in classes:
        g = wl.geom
        plan = pnp.Plan(g)
        xt = np.stack([f32(synth.ellipse_phantom(g.n, synth.phantom_seed(wl.config_id, int(i)), wl.n_ellipses))
                       for i in ids])
        d_xt = dev(xt)
        d_b = torch.empty(g.batch, g.n_views, g.n_det, device="cuda")
        plan.project(1, d_xt, d_b)
        rng = np.random.default_rng(wl.config_id)
        d_b += wl.noise_rel * float(d_b.abs().max()) * dev(rng.standard_normal((g.batch, g.n_views, g.n_det)))
        eta = [1.0 / plan.power_iter(s.factor, 60, 1e-6)[0] for s in wl.stages]
        seq = synth.schedule_sequence(wl.stages, wl.config_id)
        d_x = torch.zeros(g.batch, g.n, g.n, device="cuda")
        problems.append(dict(plan=plan, stages=wl.stages, eta=eta, seq=seq, b=d_b, x=d_x, xtrue=d_xt))
        meta.append((wl, xt, host(d_b), eta, seq))
    logs = pnp.run_many(problems, lam=0.02, tv_iters=20)
    for prob, (wl, xt, b, eta, seq), log in zip(problems, meta, logs):
        got = host(prob["x"])
        assert np.isfinite(got).all()
        assert (log[-1] > log[0]).all()
        if wl.geom.n <= 256:
            rx, _ = oracle.pnp_run(wl.geom, wl.stages, eta, seq, b[0], None, lam=0.02, tv_iters=20,
                                   momentum=True)
            assert rel(got[0], rx) < TOL_RECON, (wl.name, rel(got[0], rx))


def test_checkpoint_resume_is_bitwise_identical():
    """Stop after k iterations, keep (x_k, y_k), resume from k: the result equals
    the uninterrupted run bit for bit (deterministic kernels, same launch shapes)."""
    import torch
    g = synth.make_geometry(64, 60, 96, batch=2)
    stages = [synth.Stage(2, 4, 3), synth.Stage(1, 6, 4)]
    x, b, eta, seq = make_problem(g, stages, 13)
    plan = pnp.Plan(g)
    d_b = dev(b)
    full_x = torch.zeros(2, 64, 64, device="cuda")
    full_y = torch.zeros(2, 64, 64, device="cuda")
    pnp.run_many([dict(plan=plan, stages=stages, eta=eta, seq=seq, b=d_b, x=full_x, y=full_y)])
    k = 7
    cut = [synth.Stage(2, 4, 3), synth.Stage(1, 3, 4)]
    part_x = torch.zeros(2, 64, 64, device="cuda")
    part_y = torch.zeros(2, 64, 64, device="cuda")
    pnp.run_many([dict(plan=plan, stages=cut, eta=eta, seq=seq[:k], b=d_b, x=part_x, y=part_y)])
    pnp.run_many([dict(plan=plan, stages=stages, eta=eta, seq=seq, b=d_b, x=part_x, y=part_y, start_iter=k)])
    assert np.array_equal(host(part_x), host(full_x))
    assert np.array_equal(host(part_y), host(full_y))


def test_phase_event_timing():
    """pnp_run with PNP_RUN_KERNEL_TIMES: one timed launch per phase and
    iteration, positive device times, the same result bit for bit as a run
    without events; rejected together with graph capture."""
    import torch
    g = synth.make_geometry(64, 60, 96, batch=2)
    stages = [synth.Stage(2, 3, 5), synth.Stage(1, 4, 5)]
    x, b, eta, seq = make_problem(g, stages, 11)
    plan = pnp.Plan(g)
    plan.set_launch_shapes(tile=16)
    outs = []
    pnp.kernel_times(reset=True)
    for timed in (False, True):
        d_x = torch.zeros(g.batch, g.n, g.n, device="cuda")
        plan.run(stages, eta, seq, dev(b), d_x, kernel_times=timed)
        outs.append(host(d_x))
    assert np.array_equal(outs[0], outs[1])
    kt = pnp.kernel_times(reset=True)
    assert set(kt) == {"prep", "forward", "backward", "denoise"}
    # every iteration after the first takes y's coefficient image (2x pooled or full
    # grid; tiles of even side) from the denoiser's last launch of the iteration
    # before, unless PNP_FUSE_QUAD=0: the coefficient-image kernel runs once
    import os
    fused = os.environ.get("PNP_FUSE_QUAD", "1")[:1] != "0"
    for ph, (ms, n) in kt.items():
        assert n == (1 if fused and ph == "prep" else 7), (ph, n)
        assert ms > 0.0, ph
    assert all(n == 0 for _, n in pnp.kernel_times().values())
    with pytest.raises(pnp.PnpError):
        plan.run(stages, eta, seq, dev(b), torch.zeros(g.batch, g.n, g.n, device="cuda"),
                 kernel_times=True, graph=True)


def test_dependent_launch_changes_no_bit(tmp_path):
    """The loop kernels' programmatic dependent launch only moves launch overhead:
    a run in a process with PNP_PDL=0 (ordinary launches) gives the same bits."""
    import os
    import subprocess
    import sys
    import torch
    g = synth.make_geometry(64, 60, 96, batch=2)
    stages = [synth.Stage(2, 3, 5), synth.Stage(1, 4, 5)]
    x, b, eta, seq = make_problem(g, stages, 17)
    np.save(tmp_path / "b.npy", b)
    script = tmp_path / "run.py"
    script.write_text(f"""
import sys, numpy as np, torch
sys.path.insert(0, {os.path.dirname(os.path.dirname(os.path.abspath(__file__)))!r})
import paper_2203_07308_gb300 as pnp
from paper_2203_07308_gb300 import synth
g = synth.make_geometry(64, 60, 96, batch=2)
plan = pnp.Plan(g)
plan.set_launch_shapes(lanes=(8, 8, 0, 0), back=(4, 4, 0, 0), tile=16)
b = torch.from_numpy(np.load({str(tmp_path / "b.npy")!r}).astype(np.float32)).cuda()
x = torch.zeros(2, 64, 64, device="cuda")
plan.run([synth.Stage(2, 3, 5), synth.Stage(1, 4, 5)], {eta!r}, {list(map(int, seq))!r}, b, x)
np.save(sys.argv[1], x.cpu().numpy())
""")
    outs = []
    for pdl in ("1", "0"):
        out = tmp_path / f"x{pdl}.npy"
        env = dict(os.environ, PNP_PDL=pdl)
        subprocess.run([sys.executable, str(script), str(out)], env=env, check=True, timeout=600)
        outs.append(np.load(out))
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("tile", [0, 1, 2, 3, 4, 16])
def test_persistent_launches_give_the_same_bits(tile):
    """PNP_RUN_PERSISTENT: every phase kernel as CTAs that fit at once walking
    the work table.  Three uneven classes (sizes 48 / 64 / 96, one of them a
    batch of 9 with image-interleaved layouts) in one run_many call, every
    denoiser variant, direct and graph-captured: the iterates and PSNR logs
    equal those of the direct launches; one class against the oracle."""
    import torch
    specs = [(synth.make_geometry(48, 40, 72, batch=2), [synth.Stage(2, 2, 3), synth.Stage(1, 3, 2)]),
             (synth.make_geometry(64, 60, 96, batch=9), [synth.Stage(4, 2, 1), synth.Stage(1, 3, 4)]),
             (synth.make_geometry(96, 50, 144, batch=1), [synth.Stage(2, 3, 2), synth.Stage(1, 2, 1)])]
    base = []
    for k, (g, stages) in enumerate(specs):
        plan = pnp.Plan(g)
        if tile:
            plan.set_launch_shapes(tile=tile)
        x, b, eta, seq = make_problem(g, stages, 40 + k)
        base.append((plan, stages, eta, seq, dev(b), dev(x), x, b))
    outs = []
    for persistent, graph in ((False, False), (True, False), (True, True), (True, True)):
        probs = [dict(plan=plan, stages=st, eta=eta, seq=seq, b=b, x=torch.zeros(plan.g.batch, plan.g.n, plan.g.n,
                                                                                  device="cuda"), xtrue=xt)
                 for plan, st, eta, seq, b, xt, _, _ in base]
        logs = pnp.run_many(probs, lam=0.02, tv_iters=12, persistent=persistent, graph=graph)
        outs.append(([host(p["x"]) for p in probs], [np.asarray(l) for l in logs]))
    for run in outs[1:]:
        for k in range(len(specs)):
            assert np.array_equal(outs[0][0][k], run[0][k]), k
            assert np.array_equal(outs[0][1][k], run[1][k]), k
    plan, stages, eta, seq, _, _, x, b = base[0]
    rx, _ = oracle_runs(plan.g, stages, eta, seq, b, x, 0.02, tv_iters=12)
    assert rel(outs[1][0][0], rx) < TOL_RECON


def test_persistent_single_problem_run():
    """pnp_run with PNP_RUN_PERSISTENT on a 16-image class (batched gather,
    interleaved forward, strips): the bits of the direct launches."""
    import torch
    g = synth.make_geometry(128, 60, 192, batch=16)
    stages = [synth.Stage(2, 2, 4), synth.Stage(1, 3, 4)]
    rng = np.random.default_rng(16)
    b = dev(rng.standard_normal((16, 60, 192)))
    plan = pnp.Plan(g)
    plan.set_launch_shapes(back=((16 << 16) | (1 << 8) | 8,) * 4, tile=2)
    outs = []
    for persistent in (False, True):
        d_x = torch.zeros(16, 128, 128, device="cuda")
        plan.run(stages, [1e-4, 1e-4], [0, 1, 2, 3, 0], b, d_x, lam=0.02, tv_iters=20, persistent=persistent)
        outs.append(host(d_x))
    assert np.array_equal(outs[0], outs[1])
