"""Benchmark of the PnP-MS2G hot path on one GB300 (or N replicas under torchrun).

One step = one complete multi-stage sketched PnP reconstruction (Algorithm 1)
of a 256x256 image from 360 views x 512 bins: 20 iterations on the 2x-sketched
grid, then 80 on the full grid, each iteration one angle-subset gradient
estimate (8 interleaved subsets), the gradient step, 20 FGP iterations of the
TV-prox denoiser and the FISTA momentum.  The reported value is gradient
estimates per second (one per iteration) over the whole job.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

`--impl reference` times the FP64 CPU oracle on the host cores instead (each
step a bounded sample of the same schedule).  Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "A^T(Ax−b) gradients/s + GRay-samples/s vs HBM roofline; time-to-PSNR sketched vs full PnP"
UNIT = "gradients/s"
WORKLOAD = "c2_256"
L2_FLUSH_BYTES = 512 << 20

# DRAM bytes per launch of the backprojector at this workload, from one ncu
# capture (dram__bytes_read.sum + dram__bytes_write.sum over the 100
# backprojection launches of one step, averaged); valid only while the
# backprojector source is the one that was measured.
BACKWARD_TRAFFIC = {"bytes_per_launch": 716815,
                    "source_sha256": "da95d5be111aeb9bd6dfef2d6ffe1907fc9965197221d956979b9d331d4a2eb1",
                    "profile": "profiles/k_backward2x2_256_360x512_step.md"}


def kernel_source_sha():
    """SHA-256 of the gather backprojector's source (its table, kernel and
    launcher text), so that the stored DRAM traffic is reported only for the
    kernel it was measured on."""
    import hashlib
    with open(os.path.join(ROOT, "paper_2203_07308_gb300", "csrc", "projector.cu")) as f:
        src = f.read()
    a = src.index("struct BackTable {")
    b = src.index("// ------------------------------------------------------------------ transpose A_s^T, scatter form")
    return hashlib.sha256(src[a:b].encode()).hexdigest()


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--graph", action="store_true", help="replay a captured CUDA graph instead of direct launches")
    ap.add_argument("--no-autotune", action="store_true", help="heuristic launch shapes")
    ap.add_argument("--shapes", default=None,
                    help='pinned launch shapes instead of the autotuner, as printed in "launch_shapes", '
                         'e.g. \'{"lanes": [16, 8, 0, 0], "back": [272, 280, 0, 0], "tile": 22}\' '
                         '(for profiler runs, whose timing would mislead the autotuner)')
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched, mixed and differentiable comparisons")
    ap.add_argument("--profile", action="store_true",
                    help="only the warm-up and the timed steps (inside an NVTX range 'timed'), "
                         "for ncu: no end-to-end, time-to-PSNR or CPU legs")
    return ap.parse_args()


def dist_init(n):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    return rank, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(v, world):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            with open(self.path) as f:
                for line in f:
                    parts = [p.strip() for p in line.split(",")]
                    if len(parts) < 9:
                        continue
                    try:
                        sm.append(float(parts[1]))
                        smax = max(smax, float(parts[2]))
                    except ValueError:
                        continue
                    for nm, val in zip(names, parts[5:9]):
                        if val.lower() == "active":
                            reasons.add(nm)
            os.unlink(self.path)
        except OSError:
            pass
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax or None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------- workload
def workload():
    from paper_2203_07308_gb300 import synth
    return synth.workloads()[WORKLOAD]


def config_dict(wl, extra=None):
    g = wl.geom
    d = {"workload": f"{g.n}x{g.n} ellipse phantom, {g.n_views} views x {g.n_det} bins fan beam, "
                     "2x sketch (20 it) then full grid (80 it), 8 angle subsets, TV-FGP 20, FISTA momentum",
         "image": g.n, "views": g.n_views, "bins": g.n_det, "batch_per_gpu": g.batch,
         "schedule": [[s.factor, s.iters, s.n_subsets] for s in wl.stages],
         "iterations": sum(s.iters for s in wl.stages), "tv_iters": wl.tv_iters,
         "lambda": wl.tv_lambda, "noise_rel": wl.noise_rel,
         "l2": "flushed between timed steps (512 MiB write)"}
    if extra:
        d.update(extra)
    return d


def cpu_cores():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()


# ---------------------------------------------------------------- reference arm (FP64 oracle)
def oracle_sample_run(wl, b, x_true, eta, seq, iters_per_stage):
    """Runs the oracle on a bounded sample of the schedule (the first iterations
    of each stage); returns (seconds, gradient estimates computed)."""
    import oracle
    from paper_2203_07308_gb300 import synth
    stages = [synth.Stage(s.factor, min(s.iters, k), s.n_subsets) for s, k in zip(wl.stages, iters_per_stage)]
    sub_seq = np.concatenate([seq[sum(s.iters for s in wl.stages[:i]):][:st.iters]
                              for i, st in enumerate(stages)]) if stages else seq
    t0 = time.perf_counter()
    oracle.pnp_run(wl.geom, stages, eta, sub_seq, b, None, alpha=wl.alpha, lam=wl.tv_lambda,
                   tv_iters=wl.tv_iters, momentum=wl.momentum)
    return time.perf_counter() - t0, sum(s.iters for s in stages)


def oracle_inputs(wl):
    import oracle
    from paper_2203_07308_gb300 import synth
    g = wl.geom
    x = synth.phantom_batch(wl, 1)[0]
    w = synth.noise_draws((g.n_views, g.n_det), synth.noise_seed(wl.config_id))
    b = oracle.simulate(g, x, w, wl.noise_rel)
    seq = synth.schedule_sequence(wl.stages, synth.subset_seed(wl.config_id))
    # step sizes: the GPU arm's power iteration is not available on this leg; the
    # oracle computes its own (not timed: per-geometry set-up)
    eta = [1.0 / oracle.power_iter(g, s.factor, 15, 1e-5)[0] for s in wl.stages]
    return x, b, eta, seq


def cpu_baseline(wl, sample_iters=(2, 6)):
    os.environ.setdefault("OMP_NUM_THREADS", str(cpu_cores()))
    x, b, eta, seq = oracle_inputs(wl)
    secs, n = oracle_sample_run(wl, b, x, eta, seq, sample_iters)
    total = sum(s.iters for s in wl.stages)
    # per-operation times of the full-view operators at this size, all cores and one thread
    import oracle
    g = wl.geom
    cores = int(os.environ["OMP_NUM_THREADS"])
    per_op = {}
    for label, threads in (("all_cores", cores), ("one_thread", 1)):
        prev = oracle.set_threads(threads)
        t0 = time.perf_counter()
        sino = oracle.project(g, 1, x)
        t1 = time.perf_counter()
        oracle.backproject(g, 1, sino)
        t2 = time.perf_counter()
        oracle.grad(g, 1, x, b)
        t3 = time.perf_counter()
        oracle.set_threads(prev)
        per_op[label] = {"threads": threads, "forward_s": t1 - t0, "backproject_s": t2 - t1, "gradient_s": t3 - t2}
    return {"value": n / secs, "unit": UNIT, "cores": cores,
            "kind": "oracle", "cpu_model": cpu_model(),
            "sample": f"first {sample_iters[0]} sketched + {sample_iters[1]} full-grid iterations of the "
                      f"{total}-iteration schedule, FP64 C oracle with OpenMP over rays ({secs:.1f} s)",
            "per_op_all_views": per_op}


def cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k, _, v = line.partition(":")
                if k.strip() in ("model name", "Model"):
                    return v.strip()
                if k.strip() == "CPU part":
                    part = v.strip()
                    return {"0xd4f": "Arm Neoverse V2"}.get(part, "Arm CPU part " + part)
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def run_reference(args, rank, world):
    if rank != 0:
        return
    os.environ.setdefault("OMP_NUM_THREADS", str(cpu_cores()))
    wl = workload()
    x, b, eta, seq = oracle_inputs(wl)
    sample = (1, 3)
    for _ in range(args.warmup):
        oracle_sample_run(wl, b, x, eta, seq, sample)
    secs, n = 0.0, 0
    for _ in range(args.steps):
        s, k = oracle_sample_run(wl, b, x, eta, seq, sample)
        secs += s
        n += k
    value = n / secs
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(wl, {"step": "bounded sample: first 1 sketched + "
                                                                     "3 full-grid iterations"}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": int(os.environ["OMP_NUM_THREADS"]),
                             "kind": "oracle", "sample": "first 1 sketched + 3 full-grid iterations per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- native arm
def paper_sparse_view(plan_factory, dev, kw):
    """Sketched PnP-MS2G vs full-gradient PnP-FISTA on the paper's sparse-view
    geometry with Poisson transmission data and weighted least squares: final
    PSNR of both arms and their device times."""
    import torch
    from paper_2203_07308_gb300 import synth
    wl, i0 = synth.paper_workloads()["sparse_view"]
    g = wl.geom
    plan = plan_factory(g)
    x_true = synth.ellipse_phantom(g.n, synth.phantom_seed(wl.config_id, 0), wl.n_ellipses)
    d_xt = torch.from_numpy(x_true.astype(np.float32)).to(dev).reshape(1, g.n, g.n)
    d_ax = torch.empty(1, g.n_views, g.n_det, device=dev)
    plan.project(1, d_xt, d_ax)
    b, w = synth.poisson_transmission(d_ax.cpu().numpy()[0], i0, 5500)
    d_b = torch.from_numpy(b.astype(np.float32)).to(dev).reshape(1, g.n_views, g.n_det)
    d_w = torch.from_numpy(w.astype(np.float32)).to(dev).reshape(1, g.n_views, g.n_det)
    plan.set_weights(d_w)
    total = sum(s.iters for s in wl.stages)
    bicubic = [synth.Stage(s.factor, s.iters, s.n_subsets, kind=1) for s in wl.stages]
    arms = {"sketched": wl.stages, "sketched_bicubic": bicubic, "full": [synth.Stage(1, total, 1)]}
    out = {"setup": wl.name + ", WLS, 256x256, 228 bins",
           "schedule_sketched": [[s.factor, s.iters, s.n_subsets] for s in wl.stages],
           "iterations": total}
    pk = dict(kw)
    for name, stages in arms.items():
        eta = [1.0 / plan.power_iter(s.factor, 100, 1e-6, kind=s.kind)[0] for s in stages]
        d_x = torch.zeros(1, g.n, g.n, device=dev)
        log = plan.run(stages, eta, None, d_b, d_x, xtrue=d_xt, **pk)[:, 0]
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        plan.run(stages, eta, None, d_b, d_x.zero_(), **pk)
        ev[0].record()
        for _ in range(3):
            plan.run(stages, eta, None, d_b, d_x.zero_(), **pk)
        ev[1].record()
        torch.cuda.synchronize()
        out[name + "_final_db"] = float(log[-1])
        out[name + "_ms"] = ev[0].elapsed_time(ev[1]) / 3
    out["psnr_gap_db"] = out["full_final_db"] - out["sketched_final_db"]
    out["time_ratio_full_over_sketched"] = out["full_ms"] / out["sketched_ms"]
    return out


def l2_copy_gbs(dev, stream, mib=24, reps=50):
    """Copy bandwidth of a buffer pair that stays resident in the 129 MB L2
    (read + write bytes per second, best of three timed batches)."""
    import torch
    n = (mib << 20) // 4
    a = torch.ones(n, device=dev)
    b = torch.empty_like(a)
    for _ in range(5):
        b.copy_(a)
    best = 0.0
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            b.copy_(a)
        e1.record(stream)
        torch.cuda.synchronize()
        best = max(best, 2.0 * 4 * n * reps / (e0.elapsed_time(e1) / 1000) / 1e9)
    return best


def _simulate(plan, wl, dev, seed_offset=0):
    """x_true [B, n, n], b = A x_true + sigma w per image (GPU forward), on the device."""
    import torch
    from paper_2203_07308_gb300 import synth
    g = wl.geom
    xt = synth.phantom_batch(wl).astype(np.float32)
    d_xt = torch.from_numpy(xt).to(dev)
    d_b = torch.empty(g.batch, g.n_views, g.n_det, device=dev)
    plan.project(1, d_xt, d_b)
    w = synth.noise_draws((g.batch, g.n_views, g.n_det), synth.noise_seed(wl.config_id) + seed_offset)
    sig = wl.noise_rel * d_b.abs().amax(dim=(1, 2), keepdim=True)
    d_b += sig * torch.from_numpy(w.astype(np.float32)).to(dev)
    return d_xt, d_b


def _device_ms(fn, stream):
    import torch
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b)


def cut_schedule(stages, iters):
    """The schedule stopped after `iters` iterations: every stage kept (with its
    sketch kind and estimator), its iteration count cut, so that the step sizes
    and the subset sequence stay aligned with the full schedule."""
    cut, left = [], iters
    for st_ in stages:
        k = max(0, min(st_.iters, left))
        cut.append(dataclasses.replace(st_, iters=k))
        left -= k
    return cut


def _time_to_target(plan, stages, eta, seq, d_b, d_x, log, target, kw, stream):
    """Device time of the run cut at the first iteration whose mean PSNR reaches target."""
    hit = np.nonzero(log.mean(axis=1) >= target)[0]
    if hit.size == 0:
        return None, None
    it = int(hit[0]) + 1
    cut = cut_schedule(stages, it)
    plan.run(cut, eta, seq, d_b, d_x.zero_(), **kw)     # warm
    return _device_ms(lambda: plan.run(cut, eta, seq, d_b, d_x.zero_(), **kw), stream), it


def batched_512x16(dev, stream):
    """16 x 512^2, 720 views x 768 bins in one launch per phase: the three-stage
    sketched schedule (4x, 2x, full; 12 angle subsets) against full-gradient
    PnP-FISTA with the same iteration count, time to the full arm's final mean
    PSNR - 0.1 dB, and the sketched run's gradient estimates per second."""
    import torch
    import paper_2203_07308_gb300 as pnp
    from paper_2203_07308_gb300 import synth
    wl = synth.workloads()["c3_512x16"]
    g = wl.geom
    plan = pnp.Plan(g)
    d_xt, d_b = _simulate(plan, wl, dev)
    kw = dict(alpha=wl.alpha, lam=wl.tv_lambda, tv_iters=wl.tv_iters, momentum=wl.momentum)
    plan.autotune(wl.stages, **kw)
    eta = [1.0 / plan.power_iter(st_.factor, 100, 1e-6)[0] for st_ in wl.stages]
    seq = synth.schedule_sequence(wl.stages, synth.subset_seed(wl.config_id))
    full = synth.full_gradient_arm(wl.stages)
    d_x = torch.zeros(g.batch, g.n, g.n, device=dev)
    log_s = plan.run(wl.stages, eta, seq, d_b, d_x.zero_(), xtrue=d_xt, **kw)
    ms_s = _device_ms(lambda: plan.run(wl.stages, eta, seq, d_b, d_x.zero_(), **kw), stream)
    log_f = plan.run(full, [eta[-1]], None, d_b, d_x.zero_(), xtrue=d_xt, **kw)
    target = float(log_f[-1].mean()) - 0.1
    tts_s, it_s = _time_to_target(plan, wl.stages, eta, seq, d_b, d_x, log_s, target, kw, stream)
    tts_f, it_f = _time_to_target(plan, full, [eta[-1]], None, d_b, d_x, log_f, target, kw, stream)
    total = sum(st_.iters for st_ in wl.stages)
    return {"workload": "16 x 512x512, 720 views x 768 bins, stages (4x,24),(2x,24),(1x,72), 12 subsets",
            "sketched_run_ms": ms_s, "gradients_per_s": g.batch * total / (ms_s / 1000.0),
            "target_db": target, "sketched_final_db": float(log_s[-1].mean()),
            "full_final_db": float(log_f[-1].mean()),
            "sketched_ms": tts_s, "sketched_iters": it_s, "full_ms": tts_f, "full_iters": it_f,
            "speedup": (tts_f / tts_s) if (tts_s and tts_f) else None}


def gray_by_config(dev, stream):
    """All-view forward and backprojection throughput (GRay-samples/s: exact
    sample count / device time) for every workload size, one launch each with
    launch shapes from the autotuner."""
    import torch
    import paper_2203_07308_gb300 as pnp
    from paper_2203_07308_gb300 import synth
    wls = synth.workloads()
    cases = [("64x64, 90 x 96", wls["c1_64"].geom), ("256x256, 360 x 512", wls["c2_256"].geom),
             ("16 x 512x512, 720 x 768", wls["c3_512x16"].geom),
             ("128x128, 180 x 256", synth.make_geometry(128, 180, 256))]
    out = {}
    for name, g in cases:
        plan = pnp.Plan(g)
        plan.autotune([synth.Stage(1, 1, 1)])
        img = torch.rand(g.batch, g.n, g.n, device=dev)
        sino = torch.empty(g.batch, g.n_views, g.n_det, device=dev)
        back = torch.empty_like(img)
        samples = plan.sample_count(1) * g.batch
        plan.project(1, img, sino)
        plan.backproject(1, sino, back)
        f_ms = _device_ms(lambda: plan.project(1, img, sino), stream)
        b_ms = _device_ms(lambda: plan.backproject(1, sino, back), stream)
        out[name] = {"samples": samples, "forward_ms": f_ms, "backproject_ms": b_ms,
                     "forward_gsamples_per_s": samples / (f_ms / 1000) / 1e9,
                     "backproject_gsamples_per_s": samples / (b_ms / 1000) / 1e9}
    return out


def mixed_64(dev, stream):
    """64 instances of 128^2/180/256, 256^2/360/512 and 512^2/720/768 (seeded mix)
    in one call: every phase of every iteration one launch over the three
    classes; 50 sketched iterations each.  Also the time for every class to
    reach its full-gradient arm's final mean PSNR - 0.1 dB, sketched vs full,
    each class's schedule cut at its own first iteration on target."""
    import torch
    import paper_2203_07308_gb300 as pnp
    from paper_2203_07308_gb300 import synth
    sk, fu, n_img, iters = [], [], 0, 0
    for wl, _ids in synth.mixed_classes(64):
        g = wl.geom
        plan = pnp.Plan(g)
        d_xt, d_b = _simulate(plan, wl, dev)
        kw = dict(alpha=wl.alpha, lam=wl.tv_lambda, tv_iters=wl.tv_iters, momentum=wl.momentum)
        plan.autotune(wl.stages, **kw)
        eta = [1.0 / plan.power_iter(st_.factor, 60, 1e-6)[0] for st_ in wl.stages]
        seq = synth.schedule_sequence(wl.stages, synth.subset_seed(wl.config_id))
        full = synth.full_gradient_arm(wl.stages)
        base = dict(plan=plan, b=d_b, xtrue=d_xt)
        sk.append(dict(base, stages=wl.stages, eta=eta, seq=seq, x=torch.zeros(g.batch, g.n, g.n, device=dev)))
        fu.append(dict(base, stages=full, eta=[eta[-1]], seq=None, x=torch.zeros(g.batch, g.n, g.n, device=dev)))
        n_img += g.batch
        iters = sum(st_.iters for st_ in wl.stages)
    kw = dict(alpha=1.0, lam=0.02, tv_iters=20, momentum=True)

    def fresh(probs):                 # every run starts from x_0 = 0
        for p_ in probs:
            p_["x"].zero_()
        return probs
    untimed = [{k: v for k, v in p_.items() if k != "xtrue"} for p_ in sk]
    pnp.run_many(fresh(untimed), **kw)      # warm
    ms = _device_ms(lambda: pnp.run_many(fresh(untimed), **kw), stream)
    logs_s = pnp.run_many(fresh(sk), **kw)
    logs_f = pnp.run_many(fresh(fu), **kw)
    arms = {}
    for name, probs, logs in (("sketched", sk, logs_s), ("full", fu, logs_f)):
        cut_probs, hits = [], []
        for p_, log, lf in zip(probs, logs, logs_f):
            target = float(lf[-1].mean()) - 0.1
            hit = np.nonzero(log.mean(axis=1) >= target)[0]
            it = int(hit[0]) + 1 if hit.size else int(log.shape[0])
            hits.append(it)
            cut_probs.append(dict(plan=p_["plan"], b=p_["b"], x=p_["x"], stages=cut_schedule(p_["stages"], it),
                                  eta=p_["eta"], seq=p_["seq"]))
        run = lambda: pnp.run_many(fresh(cut_probs), **kw)      # noqa: E731
        run()
        arms[name] = {"ms": _device_ms(run, stream), "iters_per_class": hits}
    return {"workload": "64 mixed instances (seed 5308), 3 geometry classes, 50 iterations",
            "classes": [[p_["plan"].g.n, p_["plan"].g.n_views, p_["plan"].g.n_det, p_["plan"].g.batch] for p_ in sk],
            "run_ms": ms, "gradients_per_s": n_img * iters / (ms / 1000.0),
            "time_to_psnr": {"sketched": arms["sketched"], "full": arms["full"],
                             "speedup": arms["full"]["ms"] / arms["sketched"]["ms"]}}


def differentiable_256x8(dev, stream):
    """8 x 256^2, 360 x 512: 10 unrolled iterations through torch.autograd with
    the 2x sketch against the full-gradient unroll: forward + backward device
    time and the mean PSNR of x_T."""
    import torch
    import paper_2203_07308_gb300 as pnp
    from paper_2203_07308_gb300 import synth
    from paper_2203_07308_gb300.autograd import unrolled_pnp
    wl = synth.workloads()["c4_256x8"]
    g = wl.geom
    plan = pnp.Plan(g)
    d_xt, d_b = _simulate(plan, wl, dev)
    out = {"workload": "8 x 256x256, 360 views x 512 bins, 10 unrolled iterations, loss 1/2 ||x_T - x_true||^2"}
    for name, stages in (("sketched", wl.stages), ("full", [synth.Stage(1, sum(s_.iters for s_ in wl.stages), 1)])):
        eta = [1.0 / plan.power_iter(st_.factor, 60, 1e-6)[0] for st_ in stages]
        seq = synth.schedule_sequence(stages, 3)

        def fwd_bwd():
            x0 = torch.zeros(g.batch, g.n, g.n, device=dev, requires_grad=True)
            lam = torch.tensor(wl.tv_lambda, dtype=torch.float64, requires_grad=True)
            xT = unrolled_pnp(plan, stages, eta, seq, d_b, x0, lam, alpha=wl.alpha, tv_iters=wl.tv_iters)
            (0.5 * ((xT - d_xt) ** 2).sum()).backward()
            return xT.detach()
        xT = fwd_bwd()
        mse = ((xT - d_xt) ** 2).mean(dim=(1, 2)).double().cpu().numpy()
        out[name + "_fwd_bwd_ms"] = _device_ms(fwd_bwd, stream)
        out[name + "_psnr_db"] = float(np.mean(10 * np.log10(1.0 / mse)))
    out["time_ratio_full_over_sketched"] = out["full_fwd_bwd_ms"] / out["sketched_fwd_bwd_ms"]
    return out


def run_native(args, rank, world):
    import torch
    import paper_2203_07308_gb300 as pnp
    from paper_2203_07308_gb300 import build, synth

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    build.build()
    pnp.load()
    wl = workload()
    g = wl.geom
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    plan = pnp.Plan(g)

    # ---- synthetic inputs: phantom (one per rank), b = A x + sigma w (GPU forward)
    x_true = synth.ellipse_phantom(g.n, synth.phantom_seed(wl.config_id, rank), wl.n_ellipses)
    w = synth.noise_draws((g.n_views, g.n_det), synth.noise_seed(wl.config_id) + rank)
    d_xt = torch.from_numpy(x_true.astype(np.float32)).to(dev).reshape(1, g.n, g.n)
    d_b = torch.empty(1, g.n_views, g.n_det, device=dev)
    plan.project(1, d_xt, d_b)
    sigma = wl.noise_rel * float(d_b.abs().max())
    d_b += sigma * torch.from_numpy(w.astype(np.float32)).to(dev).reshape(d_b.shape)
    seq = synth.schedule_sequence(wl.stages, synth.subset_seed(wl.config_id))
    total_iters = sum(s.iters for s in wl.stages)

    # ---- per-geometry set-up (not part of a step): step sizes by power iteration
    # and the launch shapes chosen by the autotuner for this schedule
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    eta = [1.0 / plan.power_iter(s.factor, 100, 1e-6)[0] for s in wl.stages]
    setup_ms = 1000 * (time.perf_counter() - t0)
    t0 = time.perf_counter()
    if args.shapes:
        shp = json.loads(args.shapes)
        plan.set_launch_shapes(lanes=tuple(shp["lanes"]), back=tuple(shp["back"]), tile=int(shp["tile"]))
    elif not args.no_autotune:
        plan.autotune(wl.stages, alpha=wl.alpha, lam=wl.tv_lambda, tv_iters=wl.tv_iters)
    tune_ms = 1000 * (time.perf_counter() - t0)
    use_graph = args.graph

    kw = dict(alpha=wl.alpha, lam=wl.tv_lambda, tv_iters=wl.tv_iters, momentum=wl.momentum)
    d_x = torch.zeros(1, g.n, g.n, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def step():
        d_x.zero_()
        plan.run(wl.stages, eta, seq, d_b, d_x, graph=use_graph, **kw)

    launches_setup = pnp.launch_count()
    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    barrier(world)

    if args.profile:
        torch.cuda.nvtx.range_push("timed")
        for _ in range(args.steps):
            step()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        if rank == 0:
            print(json.dumps({"profile": True, "steps": args.steps, "launches_per_step":
                              (pnp.launch_count() - launches_setup) // (args.steps + max(args.warmup, 3))}))
        return

    # ---- timed region: K steps, L2 flushed before each, device time by CUDA events
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    launches0 = pnp.launch_count()
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        barrier(world)
        for k in range(args.steps):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            plan.run(wl.stages, eta, seq, d_b, d_x.zero_(), graph=use_graph, **kw)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        barrier(world)
    launches = pnp.launch_count() - launches0

    # ---- the same K steps again with a CUDA event pair on the run's stream
    # around every phase launch: each kernel's live launch durations.  (The
    # events cost ~2 us of front-end time each, so the step above carries none.)
    pnp.kernel_times(reset=True)
    ev_ph = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
             for _ in range(args.steps)]
    if not use_graph:
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.fill_(float(k))
            ev_ph[k][0].record(stream)
            plan.run(wl.stages, eta, seq, d_b, d_x.zero_(), kernel_times=True, **kw)
            ev_ph[k][1].record(stream)
        torch.cuda.synchronize()
    phases = pnp.kernel_times(reset=True)
    ms_with_events = (float(np.mean([a.elapsed_time(b) for a, b in ev_ph])) if not use_graph else None)
    # d_x.zero_() is a PyTorch fill inside the region: not counted as ours
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = allmax(sum(step_ms), world)
    value = world * total_iters * args.steps / (total_ms / 1000.0)

    # ---- the same step in the other launch mode (graph replay vs direct), for comparison
    other = []
    for k in range(5):
        flush.fill_(3.0)
        a_, b2_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a_.record(stream)
        plan.run(wl.stages, eta, seq, d_b, d_x.zero_(), graph=not use_graph, **kw)
        b2_.record(stream)
        torch.cuda.synchronize()
        if k >= 2:
            other.append(a_.elapsed_time(b2_))
    other_ms = float(np.median(other))

    # ---- per-kernel timing of the projector pair (events on the launching stream)
    def timed(fn, reps=20):
        fn()
        torch.cuda.synchronize()
        es = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for a, b in es:
            flush.fill_(1.0)
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize()
        return float(np.mean([a.elapsed_time(b) for a, b in es]))

    res = torch.empty(1, g.n_views, g.n_det, device=dev)
    img = torch.empty(1, g.n, g.n, device=dev)
    fwd_ms = timed(lambda: plan.project(1, d_xt, res, d_b))
    back_ms = timed(lambda: plan.backproject(1, res, img))
    grad_ms = timed(lambda: plan.full_grad(d_xt, d_b, img))
    samples_full = plan.sample_count(1)
    gray_fwd = samples_full / (fwd_ms / 1000) / 1e9
    gray_back = samples_full / (back_ms / 1000) / 1e9

    # ---- time-to-PSNR: sketched schedule vs full-gradient PnP-FISTA, same data
    full_arm = synth.full_gradient_arm(wl.stages)
    eta_full = [eta[[s.factor for s in wl.stages].index(1)]]
    d_x.zero_()
    log_s = plan.run(wl.stages, eta, seq, d_b, d_x, xtrue=d_xt, **kw)[:, 0]
    d_x.zero_()
    log_f = plan.run(full_arm, eta_full, None, d_b, d_x, xtrue=d_xt, **kw)[:, 0]
    target = float(log_f[-1]) - 0.1

    def time_to(stages, etas, sq, log):
        hit = np.nonzero(log >= target)[0]
        if hit.size == 0:
            return None, None
        it = int(hit[0]) + 1
        cut = cut_schedule(stages, it)

        def go():
            d_x.zero_()
            plan.run(cut, etas, sq, d_b, d_x, **kw)
        return timed(go, reps=5), it

    tts_s, it_s = time_to(wl.stages, eta, seq, log_s)
    tts_f, it_f = time_to(full_arm, eta_full, None, log_f)

    # ---- the paper's sparse-view set-up (Sec. 3: 90 views, 228 bins, Poisson
    # data with I0 = 10^5.5, two sketch stages m_1 = d/16 then m_2 = d/4,
    # Option 1) against full-gradient PnP-FISTA with the same iteration count
    paper = paper_sparse_view(plan_factory=pnp.Plan, dev=dev, kw=kw)
    extras = {}
    if not args.no_extras:
        extras = {"batched_512x16": batched_512x16(dev, stream), "mixed_64": mixed_64(dev, stream),
                  "differentiable_256x8": differentiable_256x8(dev, stream),
                  "gray_by_config": gray_by_config(dev, stream)}

    # ---- end to end through the C ABI with host buffers (pinned), copies timed
    h_b = torch.empty(d_b.shape, dtype=torch.float32, pin_memory=True)
    h_b.copy_(d_b)
    h_x0 = torch.zeros(d_x.shape, dtype=torch.float32, pin_memory=True)
    h_out = torch.empty(d_x.shape, dtype=torch.float32, pin_memory=True)
    d_b2 = torch.empty_like(d_b)
    e2e_ms = []
    for k in range(args.steps + 1):
        flush.fill_(2.0)
        a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        d_b2.copy_(h_b, non_blocking=True)
        d_x.copy_(h_x0, non_blocking=True)
        plan.run(wl.stages, eta, seq, d_b2, d_x, graph=use_graph, **kw)
        h_out.copy_(d_x, non_blocking=True)
        b_.record(stream)
        torch.cuda.synchronize()
        if k > 0:
            e2e_ms.append(a.elapsed_time(b_))
    e2e_total = allmax(sum(e2e_ms), world)
    e2e_value = world * total_iters * len(e2e_ms) / (e2e_total / 1000.0)

    # ---- roofline of the dominant projector kernel
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    sm_mhz = 2070.0
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    # FP32 issue peak: 128 lanes/SM/clock, FMA = 2 FLOP
    alu_peak = n_sm * 128 * 2 * sm_mhz * 1e6 / 1e12
    # algorithmic work per backprojected sample: 4 bilinear taps, each
    # hat(dx) hat(dy) r: 2 position FMA + 2 |.| + 2 (1-.) + 1 mul + 1 FMA = 8 FLOP per tap
    # (the forward: position 2 FMA, 3 FMA interpolation, accumulate = 11 FLOP)
    FLOP_BACK, FLOP_FWD = 4 * 8, 4 + 3 * 2 + 1
    # samples of every iteration's subset projection at its level, in step order
    counts = {}
    samples_step = 0
    it_cursor = 0
    for st_ in wl.stages:
        for _ in range(st_.iters):
            p_ = int(seq[it_cursor]) if st_.n_subsets > 1 else 0
            key = (st_.factor, p_, st_.n_subsets)
            if key not in counts:
                counts[key] = plan.sample_count(*key)
            samples_step += counts[key]
            it_cursor += 1
    ph_ms = {k: v[0] for k, v in phases.items()}
    ph_n = {k: v[1] for k, v in phases.items()}
    if ph_n["backward"] > 0:
        dominant = max(("backward", "forward"), key=lambda k: ph_ms[k])
        flop = samples_step * (FLOP_BACK if dominant == "backward" else FLOP_FWD) * args.steps
        ach = flop / (ph_ms[dominant] / 1000) / 1e12
        kname = "k_backward2x2 (A^T, U and the step)" if dominant == "backward" else "k_forward (A S y - b)"
        avg_us = 1000 * ph_ms[dominant] / ph_n[dominant]
        timing_src = (f"CUDA event pair around each of the {ph_n[dominant]} launches of the K timed steps "
                      f"re-run with phase events, mean {avg_us:.2f} us per launch")
    else:   # graph replay: phases are not bracketed; the all-views launch timed alone
        dominant = "backward" if back_ms >= fwd_ms else "forward"
        ach = samples_full * (FLOP_BACK if dominant == "backward" else FLOP_FWD) / (
            (back_ms if dominant == "backward" else fwd_ms) / 1000) / 1e12
        kname = "k_backward2x2 all views" if dominant == "backward" else "k_forward all views"
        timing_src = "CUDA events around the all-views launch timed alone"
    # the forward against the memory level it streams its taps from: 16 B of
    # coefficients per sample from L1/L2 (the level image is L2-resident), vs an
    # L2-resident copy (2 x 24 MiB) measured here
    l2_gbs = l2_copy_gbs(dev, stream)
    roof_fwd = None
    if ph_n["forward"] > 0:
        gbs = 16.0 * samples_step * args.steps / (ph_ms["forward"] / 1000) / 1e9
        roof_fwd = {"kernel": "k_forward (A S y - b)", "bound": "l2", "achieved": gbs, "peak": l2_gbs,
                    "unit": "GB/s", "frac": gbs / l2_gbs, "bytes_per_sample": 16,
                    "peak_source": "L2-resident device copy of 2 x 24 MiB, read + write bytes, measured here"}
    traffic = None
    if dominant == "backward" and kernel_source_sha() == BACKWARD_TRAFFIC["source_sha256"]:
        traffic = BACKWARD_TRAFFIC["bytes_per_launch"]
    roof = {"kernel": kname, "bound": "alu", "achieved": ach, "peak": alu_peak, "unit": "TFLOP/s",
            "frac": ach / alu_peak, "traffic": traffic,
            "flop_per_sample": FLOP_BACK if dominant == "backward" else FLOP_FWD,
            "samples_per_step": samples_step, "timing": timing_src,
            "peak_source": f"{n_sm} SMs x 128 FP32 lanes x 2 FLOP x {sm_mhz:.0f} MHz (derived)",
            "hbm_gbs_measured_peak": peaks.get("hbm_gbs")}

    clocks = clk.summary()
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": config_dict(wl, {"parallelism": f"replicas x{world}" if world > 1 else "single GPU"}),
            "clocks": clocks,
            "e2e": {"value": e2e_value, "unit": UNIT,
                    "h2d_bytes_per_step": int(d_b.numel() * 4 + d_x.numel() * 4),
                    "d2h_bytes_per_step": int(d_x.numel() * 4)},
            "gpu_launches": int(launches),
            "roofline": roof,
            "roofline_forward": roof_fwd,
            "kernels_ms": {"forward_all_views": fwd_ms, "backproject_all_views": back_ms,
                           "full_gradient": grad_ms},
            "gray_samples_per_s": {"forward": gray_fwd, "backproject": gray_back,
                                   "samples_per_projection": samples_full},
            "full_gradients_per_s": 1000.0 / grad_ms,
            "time_to_psnr": {"target_db": target, "full_final_db": float(log_f[-1]),
                             "sketched_final_db": float(log_s[-1]),
                             "sketched_ms": tts_s, "sketched_iters": it_s,
                             "full_ms": tts_f, "full_iters": it_f,
                             "speedup": (tts_f / tts_s) if (tts_s and tts_f) else None},
            "paper_sparse_view": paper,
            **extras,
            "setup_ms_power_iteration": setup_ms,
            "setup_ms_autotune": tune_ms,
            "launch_mode": "CUDA graph captured once, replayed per step" if use_graph else "direct launches",
            "launch_shapes": plan.launch_shapes(),
            "ms_per_step_other_launch_mode": other_ms,
            "ms_per_step_with_phase_events": ms_with_events,
            "phase_ms_per_step": {k: v / args.steps for k, v in ph_ms.items()},
            "phase_launches_per_step": {k: v // args.steps for k, v in ph_n.items()},
            "step_ms_all": step_ms}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl)
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world = dist_init(args.gpus)
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_native(args, rank, world)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
