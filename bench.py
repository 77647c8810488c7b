"""Benchmark of the PnP-MS2G hot path on one GB300 (or N replicas under torchrun).

One step = one complete multi-stage sketched PnP reconstruction (Algorithm 1)
of a batch of 16 images of 512x512 from 720 views x 768 bins, all 16 in one
launch per phase: 24 iterations on the 4x-sketched grid, 24 on the 2x grid,
then 72 on the full grid, each iteration one angle-subset gradient estimate
(12 interleaved subsets) per image, the gradient step, 20 FGP iterations of the
TV-prox denoiser and the FISTA momentum.  The reported value is gradient
estimates per second (one per image and iteration) over the whole job.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

`--impl reference` times the FP64 CPU oracle on the host cores instead (each
step a bounded sample of the same schedule on one image).  Prints one JSON
line (rank 0).
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
UNIT = "gradient_estimates/s"
WORKLOAD = "c3_512x16"
L2_FLUSH_BYTES = 512 << 20

# Algorithmic work per projected sample (the same for the forward and the
# backprojection): 4 bilinear taps of 4 B (16 B gathered) and about 12 FP32
# operations (2 FMA for the position, 2 floor/fraction, 3 lerps, 1 accumulate).
FLOP_PER_SAMPLE = 12
BYTES_PER_SAMPLE = 16

# Algorithmic work per pixel and FGP iteration of the TV-prox denoiser (Beck &
# Teboulle's FGP): L(r) 3 adds, z - lambda L 1 FMA, two differences, two dual
# FMAs, |a|^2 (mul + FMA), projection (compare, rsqrt, 2 mul), momentum (2 x
# (sub + FMA)): 24 FP32 operations.
FLOP_PER_PIXEL_ITER = 24

# DRAM bytes per unit of each kernel at the headline workload, from one ncu
# capture (dram__bytes_read.sum + dram__bytes_write.sum, cold caches), valid only
# while the kernel's source is the one that was measured (else null).  Units: one
# launch of the projector kernels (the forward's figure weighted over the
# schedule's 24 / 24 / 72 launches at the 4x / 2x / full levels, whose captured
# launches move 8.3 / 21.0 / 81.7 MB), one denoise (two launches) of the FGP strips.
KERNEL_TRAFFIC = {
    "backward": {"bytes_per_unit": 20119040, "unit": "launch", "source": "projector.cu",
                 "begin": "struct BackTable {",
                 "end": "// ------------------------------------------------------------------ transpose A_s^T from a stored table",
                 "sha256": "2f8fa2711e611cb611aff4100728e2c28dd89026404b31e1d60ae795b95014e8",
                 "profile": "profiles/k_backward_batch_512x16_720x768.md"},
    "forward": {"bytes_per_unit": 54855782, "unit": "launch", "source": "projector.cu",
                "begin": "// Forward projector on an image-interleaved coefficient image.",
                "end": "// ------------------------------------------------------------------ transpose A_s^T\n// Pixel-driven gather.",
                "sha256": "8200a95fafaaef7a9f5ffe6ae83b6eeeea278d83369f712a07bd979f85925580",
                 "profile": "profiles/k_forward_il_512x16_720x768.md"},
    "denoise": {"bytes_per_unit": 126000128, "unit": "denoise (two launches)", "source": "tv.cu",
                "begin": "// ------------------------------------------------------------------ register-resident FGP strips",
                "end": "inline cudaError_t counted(cudaError_t e = cudaGetLastError())",
                "sha256": "e20a75d6f0fd5609643ab084cd3afa299298d80e8eb1646c7c4f2756ace31cd4",
                 "profile": "profiles/k_tv_strip_512x16.md"},
}


def kernel_source_sha(kind):
    """SHA-256 of a kernel's source text (the section between two markers of its
    file), so that a stored DRAM traffic is reported only for the kernel it was
    measured on."""
    import hashlib
    k = KERNEL_TRAFFIC[kind]
    with open(os.path.join(ROOT, "paper_2203_07308_gb300", "csrc", k["source"])) as f:
        src = f.read()
    a = src.index(k["begin"])
    b = src.index(k["end"].replace("\\n", "\n"), a)
    return hashlib.sha256(src[a:b].encode()).hexdigest()


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--graph", action="store_true", help="replay a captured CUDA graph instead of direct launches")
    ap.add_argument("--no-autotune", action="store_true", help="heuristic launch shapes")
    ap.add_argument("--shapes", default=None,
                    help='pinned launch shapes instead of the autotuner, as printed in "launch_shapes", '
                         'e.g. \'{"lanes": [16, 8, 4, 0], "back": [272, 280, 264, 0], "tile": 22}\' '
                         '(for profiler runs, whose timing would mislead the autotuner)')
    ap.add_argument("--workload", default=WORKLOAD, help="synth.workloads() key of the timed step")
    ap.add_argument("--eta", type=float, default=None,
                    help="one fixed step size for every stage instead of the library's eta_k = 1/L_k "
                         "(profiler runs: kernel times do not depend on it)")
    ap.add_argument("--stage-iters", type=int, default=None,
                    help="cut every stage of the schedule to this many iterations (profiler captures of "
                         "single kernels, so that few launches precede the captured one)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the 256^2, mixed, differentiable and paper-geometry comparisons")
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
def workload(key=WORKLOAD):
    from paper_2203_07308_gb300 import synth
    return synth.workloads()[key]


def describe_schedule(wl):
    parts = [f"{s.factor}x ({s.iters} it)" if s.factor > 1 else f"full grid ({s.iters} it)" for s in wl.stages]
    P = max(s.n_subsets for s in wl.stages)
    return ", then ".join(parts) + (f", {P} angle subsets" if P > 1 else "")


def config_dict(wl, extra=None):
    g = wl.geom
    d = {"workload": f"{g.batch} x {g.n}x{g.n} ellipse phantoms, {g.n_views} views x {g.n_det} bins fan beam, "
                     f"{describe_schedule(wl)}, TV-FGP {wl.tv_iters}, FISTA momentum, "
                     f"noise {wl.noise_rel * 100:g}% of max|Ax|",
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


def sample_schedule(stages, per_stage):
    """The first `per_stage[k]` iterations of every stage (the CPU legs' bounded
    sample) and the positions of those iterations in the full schedule."""
    out, pos, start = [], [], 0
    for st_, k in zip(stages, per_stage):
        m = min(st_.iters, k)
        out.append(dataclasses.replace(st_, iters=m))
        pos.extend(range(start, start + m))
        start += st_.iters
    return out, np.asarray(pos, dtype=np.int64)


# ---------------------------------------------------------------- reference arm (FP64 oracle)
def oracle_inputs(wl):
    """One image of the workload, its data b = A x + sigma w (oracle forward) and
    step sizes for the oracle's sampled iterations.  The step sizes come from 3
    power iterations of the oracle on angle subset 0 of P, scaled by P (the work
    of an iteration does not depend on eta, so an estimate keeps the sample
    well scaled without a full-operator power iteration on the CPU)."""
    import oracle
    from paper_2203_07308_gb300 import synth
    g = dataclasses.replace(wl.geom, batch=1)
    x = synth.phantom_batch(wl, 1)[0]
    w = synth.noise_draws((g.n_views, g.n_det), synth.noise_seed(wl.config_id))
    b = oracle.simulate(g, x, w, wl.noise_rel)
    seq = synth.schedule_sequence(wl.stages, synth.subset_seed(wl.config_id))
    eta = []
    for s in wl.stages:
        P = max(s.n_subsets, 1)
        gs = g if P == 1 else dataclasses.replace(g, n_views=len(range(0, g.n_views, P)),
                                                 angle_span=g.angle_span * len(range(0, g.n_views, P)) * P / g.n_views)
        L, _ = oracle.power_iter(gs, s.factor, 3, 0.0)
        eta.append(1.0 / (L * P))
    return g, x, b, eta, seq


def oracle_sample_run(wl, g, b, eta, seq, per_stage):
    """The oracle on a bounded sample of the schedule (the first iterations of
    each stage, one image); returns (seconds, gradient estimates computed)."""
    import oracle
    stages, pos = sample_schedule(wl.stages, per_stage)
    t0 = time.perf_counter()
    oracle.pnp_run(g, stages, eta, seq[pos], b, None, alpha=wl.alpha, lam=wl.tv_lambda,
                   tv_iters=wl.tv_iters, momentum=wl.momentum)
    return time.perf_counter() - t0, int(pos.size)


def sample_text(wl, per_stage, secs=None):
    parts = [f"{min(s.iters, k)} at {s.factor}x" for s, k in zip(wl.stages, per_stage)]
    t = f" ({secs:.1f} s)" if secs is not None else ""
    return (f"first iterations of each stage ({', '.join(parts)}) of the {sum(s.iters for s in wl.stages)}-"
            f"iteration schedule, one {wl.geom.n}x{wl.geom.n} image, FP64 C oracle, OpenMP over rays and view "
            f"chunks{t}")


def cpu_baseline(wl, per_stage=(4, 4, 6)):
    os.environ.setdefault("OMP_NUM_THREADS", str(cpu_cores()))
    import oracle
    g, x, b, eta, seq = oracle_inputs(wl)
    cores = int(os.environ["OMP_NUM_THREADS"])
    oracle.set_threads(cores)
    secs, n = oracle_sample_run(wl, g, b, eta, seq, per_stage[:len(wl.stages)])
    # per-operation times of one 60-view subset at the full grid, all cores and one thread
    P = max(s.n_subsets for s in wl.stages)
    per_op = {}
    for label, threads in (("all_cores", cores), ("one_thread", 1)):
        prev = oracle.set_threads(threads)
        t0 = time.perf_counter()
        r = oracle.project(g, 1, x, b, 0, P)
        t1 = time.perf_counter()
        oracle.backproject(g, 1, r, 0, P)
        t2 = time.perf_counter()
        oracle.set_threads(prev)
        per_op[label] = {"threads": threads, "forward_s": t1 - t0, "backproject_s": t2 - t1}
    return {"value": n / secs, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": cpu_model(),
            "sample": sample_text(wl, per_stage, secs),
            "per_op_subset_full_grid": per_op}


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
    import oracle
    wl = workload(args.workload)
    g, x, b, eta, seq = oracle_inputs(wl)
    cores = int(os.environ["OMP_NUM_THREADS"])
    oracle.set_threads(cores)
    sample = (1,) * len(wl.stages)
    for _ in range(args.warmup):
        oracle_sample_run(wl, g, b, eta, seq, sample)
    secs, n = 0.0, 0
    for _ in range(args.steps):
        s, k = oracle_sample_run(wl, g, b, eta, seq, sample)
        secs += s
        n += k
    value = n / secs
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(wl),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "each step: " + sample_text(wl, sample)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- native arm: helpers
def _device_ms(fn, stream):
    import torch
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b)


def _simulate(plan, wl, dev, seed_offset=0):
    """x_true [B, n, n], b = A x_true + sigma w per image (GPU forward), on the device."""
    import torch
    from paper_2203_07308_gb300 import synth
    g = wl.geom
    xt = np.stack([synth.ellipse_phantom(g.n, synth.phantom_seed(wl.config_id, i) + 100 * seed_offset,
                                         wl.n_ellipses) for i in range(g.batch)]).astype(np.float32)
    d_xt = torch.from_numpy(xt).to(dev)
    d_b = torch.empty(g.batch, g.n_views, g.n_det, device=dev)
    plan.project(1, d_xt, d_b)
    w = synth.noise_draws((g.batch, g.n_views, g.n_det), synth.noise_seed(wl.config_id) + seed_offset)
    sig = wl.noise_rel * d_b.abs().amax(dim=(1, 2), keepdim=True)
    d_b += sig * torch.from_numpy(w.astype(np.float32)).to(dev)
    return d_xt, d_b


def _time_to_target(plan, stages, eta, seq, d_b, d_x, log, target, kw, stream):
    """Device time of the run cut at the first iteration whose mean PSNR reaches target."""
    hit = np.nonzero(log.mean(axis=1) >= target)[0]
    if hit.size == 0:
        return None, None
    it = int(hit[0]) + 1
    cut = cut_schedule(stages, it)
    plan.run(cut, eta, seq, d_b, d_x.zero_(), **kw)     # warm
    return _device_ms(lambda: plan.run(cut, eta, seq, d_b, d_x.zero_(), **kw), stream), it


def onchip_peaks():
    import paper_2203_07308_gb300 as pnp
    return pnp.onchip_bandwidth()


def rooflines(samples_step, pixel_iters_step, steps, ph_ms, ph_n, n_sm, clock_mhz, onchip):
    """Per-kernel rooflines of the projector pair and the denoiser from their live
    launch durations (phase events) and their algorithmic work: per projected
    sample 12 FP32 operations and 16 B of taps, per pixel and FGP iteration 24
    FP32 operations."""
    alu_peak = n_sm * 128 * 2 * clock_mhz * 1e6 / 1e12      # FP32 TFLOP/s: 128 lanes x FMA per SM per clock
    out = {}
    for ph, kname in (("backward", "k_backward_batch (A_s^T, U and the gradient step)"),
                      ("forward", "k_forward_il (A_s S y - b)"),
                      ("denoise", "k_tv_strip (TV-prox by FGP, relaxation, momentum)")):
        if ph_n.get(ph, 0) <= 0 or ph_ms.get(ph, 0.0) <= 0.0:
            continue
        secs = ph_ms[ph] / 1000.0
        if ph == "denoise":
            flop = FLOP_PER_PIXEL_ITER * pixel_iters_step * steps
            tflops = flop / secs / 1e12
            out[ph] = {"kernel": kname, "units": ph_n[ph], "unit": "denoise (20 FGP iterations, two launches)",
                       "mean_unit_us": 1000.0 * ph_ms[ph] / ph_n[ph],
                       "gpixel_iters_per_s": pixel_iters_step * steps / secs / 1e9,
                       "alu": {"achieved": tflops, "peak": alu_peak, "unit": "TFLOP/s", "frac": tflops / alu_peak}}
            continue
        samples = samples_step * steps
        tflops = FLOP_PER_SAMPLE * samples / secs / 1e12
        gbs = BYTES_PER_SAMPLE * samples / secs / 1e9
        out[ph] = {"kernel": kname, "units": ph_n[ph], "unit": "launch",
                   "mean_unit_us": 1000.0 * ph_ms[ph] / ph_n[ph],
                   "gsamples_per_s": samples / secs / 1e9,
                   "alu": {"achieved": tflops, "peak": alu_peak, "unit": "TFLOP/s", "frac": tflops / alu_peak},
                   "l1": {"achieved": gbs, "peak": onchip["l1_gbs"], "unit": "GB/s", "frac": gbs / onchip["l1_gbs"]},
                   "l2": {"achieved": gbs, "peak": onchip["l2_gbs"], "unit": "GB/s", "frac": gbs / onchip["l2_gbs"]}}
    return out, alu_peak


def step_samples(plan, wl, seq):
    """Exact projected samples of one step: sum over the schedule's iterations of
    the subset's sample count at the iteration's level, times the batch."""
    counts, total, i = {}, 0.0, 0
    for st_ in wl.stages:
        for _ in range(st_.iters):
            p_ = int(seq[i]) if st_.n_subsets > 1 else 0
            key = (st_.factor, p_, st_.n_subsets)
            if key not in counts:
                counts[key] = plan.sample_count(*key)
            total += counts[key]
            i += 1
    return total * wl.geom.batch


# ---------------------------------------------------------------- extras
def paper_sparse_view(dev, kw):
    """Sketched PnP-MS2G vs full-gradient PnP-FISTA on the paper's sparse-view
    geometry with Poisson transmission data and weighted least squares: final
    PSNR of both arms and their device times."""
    import torch
    import paper_2203_07308_gb300 as pnp
    from paper_2203_07308_gb300 import synth
    wl, i0 = synth.paper_workloads()["sparse_view"]
    g = wl.geom
    plan = pnp.Plan(g)
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
    for name, stages in arms.items():
        d_x = torch.zeros(1, g.n, g.n, device=dev)
        log = plan.run(stages, None, None, d_b, d_x, xtrue=d_xt, **kw)[:, 0]
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        plan.run(stages, None, None, d_b, d_x.zero_(), **kw)
        ev[0].record()
        for _ in range(3):
            plan.run(stages, None, None, d_b, d_x.zero_(), **kw)
        ev[1].record()
        torch.cuda.synchronize()
        out[name + "_final_db"] = float(log[-1])
        out[name + "_ms"] = ev[0].elapsed_time(ev[1]) / 3
    out["psnr_gap_db"] = out["full_final_db"] - out["sketched_final_db"]
    out["time_ratio_full_over_sketched"] = out["full_ms"] / out["sketched_ms"]
    return out


def gray_by_config(dev, stream):
    """All-view forward and backprojection throughput (GRay-samples/s: exact
    sample count / device time) for every workload size, one launch each with
    launch shapes from the autotuner."""
    import torch
    import paper_2203_07308_gb300 as pnp
    from paper_2203_07308_gb300 import synth
    wls = synth.workloads()
    cases = [("64x64, 90 x 96", wls["c1_64"].geom), ("256x256, 360 x 512", wls["c2_256"].geom),
             ("8 x 256x256, 360 x 512", wls["c4_256x8"].geom),
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
        f_ms = min(_device_ms(lambda: plan.project(1, img, sino), stream) for _ in range(3))
        b_ms = min(_device_ms(lambda: plan.backproject(1, sino, back), stream) for _ in range(3))
        out[name] = {"samples": samples, "forward_ms": f_ms, "backproject_ms": b_ms,
                     "forward_gsamples_per_s": samples / (f_ms / 1000) / 1e9,
                     "backproject_gsamples_per_s": samples / (b_ms / 1000) / 1e9,
                     "launch_shapes": plan.launch_shapes()}
    return out


def single_256(dev, stream, args):
    """The single-image 256^2 / 360 x 512 workload (2x sketch for 20 iterations,
    then the full grid for 80, 8 subsets), with the stored gather table
    registered: gradient estimates per second of the whole schedule and
    time-to-PSNR against full-gradient PnP-FISTA."""
    import torch
    import paper_2203_07308_gb300 as pnp
    from paper_2203_07308_gb300 import synth
    wl = synth.workloads()["c2_256"]
    g = wl.geom
    plan = pnp.Plan(g, gather_table=True)          # the autotuner also times the stored-table gather
    d_xt, d_b = _simulate(plan, wl, dev)
    kw = dict(alpha=wl.alpha, lam=wl.tv_lambda, tv_iters=wl.tv_iters, momentum=wl.momentum)
    plan.autotune(wl.stages, **kw)
    eta = plan.step_sizes(wl.stages)
    seq = synth.schedule_sequence(wl.stages, synth.subset_seed(wl.config_id))
    d_x = torch.zeros(1, g.n, g.n, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    for _ in range(3):
        plan.run(wl.stages, eta, seq, d_b, d_x.zero_(), **kw)
    ms = []
    for k in range(10):
        flush.fill_(float(k))
        ms.append(_device_ms(lambda: plan.run(wl.stages, eta, seq, d_b, d_x.zero_(), **kw), stream))
    total = sum(s.iters for s in wl.stages)
    full = synth.full_gradient_arm(wl.stages)
    eta_full = plan.step_sizes(full)
    log_s = plan.run(wl.stages, eta, seq, d_b, d_x.zero_(), xtrue=d_xt, **kw)
    log_f = plan.run(full, eta_full, None, d_b, d_x.zero_(), xtrue=d_xt, **kw)
    target = float(log_f[-1].mean()) - 0.1
    tts_s, it_s = _time_to_target(plan, wl.stages, eta, seq, d_b, d_x, log_s, target, kw, stream)
    tts_f, it_f = _time_to_target(plan, full, eta_full, None, d_b, d_x, log_f, target, kw, stream)
    return {"workload": "256x256, 360 views x 512 bins, 2x (20 it) then full grid (80 it), 8 subsets",
            "ms_per_run": float(np.mean(ms)), "gradient_estimates_per_s": total / (float(np.mean(ms)) / 1000.0),
            "launch_shapes": plan.launch_shapes(), "gather_table_bytes": int(plan.table.numel()),
            "time_to_psnr": {"target_db": target, "sketched_ms": tts_s, "sketched_iters": it_s,
                             "full_ms": tts_f, "full_iters": it_f,
                             "speedup": (tts_f / tts_s) if (tts_s and tts_f) else None}}


def mixed_64(dev, stream):
    """64 instances of 128^2/180/256, 256^2/360/512 and 512^2/720/768 (seeded mix)
    in one call, replayed from a captured CUDA graph: every phase of every
    iteration one launch over the three classes; 50 sketched iterations each.
    Also the time for every class to reach its full-gradient arm's final mean
    PSNR - 0.1 dB, sketched vs full, each class's schedule cut at its own first
    iteration on target."""
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
        seq = synth.schedule_sequence(wl.stages, synth.subset_seed(wl.config_id))
        full = synth.full_gradient_arm(wl.stages)
        eta = plan.step_sizes(wl.stages)
        eta_f = plan.step_sizes(full)
        base = dict(plan=plan, b=d_b, xtrue=d_xt)
        sk.append(dict(base, stages=wl.stages, eta=eta, seq=seq, x=torch.zeros(g.batch, g.n, g.n, device=dev)))
        fu.append(dict(base, stages=full, eta=eta_f, seq=None, x=torch.zeros(g.batch, g.n, g.n, device=dev)))
        n_img += g.batch
        iters = sum(st_.iters for st_ in wl.stages)
    kw = dict(alpha=1.0, lam=0.02, tv_iters=20, momentum=True)

    def fresh(probs):                 # every run starts from x_0 = 0
        for p_ in probs:
            p_["x"].zero_()
        return probs
    untimed = [{k: v for k, v in p_.items() if k != "xtrue"} for p_ in sk]
    pnp.run_many(fresh(untimed), graph=True, **kw)      # capture
    pnp.run_many(fresh(untimed), graph=True, **kw)      # warm replay
    ms_graph = _device_ms(lambda: pnp.run_many(fresh(untimed), graph=True, **kw), stream)
    ms_direct = _device_ms(lambda: pnp.run_many(fresh(untimed), **kw), stream)
    # every phase kernel in its persistent form (CTAs that fit at once walk the work table)
    pnp.run_many(fresh(untimed), graph=True, persistent=True, **kw)
    pnp.run_many(fresh(untimed), graph=True, persistent=True, **kw)
    ms_persistent = _device_ms(lambda: pnp.run_many(fresh(untimed), graph=True, persistent=True, **kw), stream)
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
        run = lambda: pnp.run_many(fresh(cut_probs), graph=True, **kw)      # noqa: E731
        run()
        run()
        arms[name] = {"ms": _device_ms(run, stream), "iters_per_class": hits}
    return {"workload": "64 mixed instances (seed 5308), 3 geometry classes, 50 iterations",
            "classes": [[p_["plan"].g.n, p_["plan"].g.n_views, p_["plan"].g.n_det, p_["plan"].g.batch] for p_ in sk],
            "launch_mode": "CUDA graph captured once, replayed",
            "run_ms": ms_graph, "run_ms_direct_launches": ms_direct, "run_ms_persistent_graph": ms_persistent,
            "gradient_estimates_per_s": n_img * iters / (ms_graph / 1000.0),
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
        seq = synth.schedule_sequence(stages, 3)

        def fwd_bwd():
            x0 = torch.zeros(g.batch, g.n, g.n, device=dev, requires_grad=True)
            lam = torch.tensor(wl.tv_lambda, dtype=torch.float64, requires_grad=True)
            xT = unrolled_pnp(plan, stages, None, seq, d_b, x0, lam, alpha=wl.alpha, tv_iters=wl.tv_iters)
            (0.5 * ((xT - d_xt) ** 2).sum()).backward()
            return xT.detach()
        xT = fwd_bwd()
        mse = ((xT - d_xt) ** 2).mean(dim=(1, 2)).double().cpu().numpy()
        # a host-driven loop (autograd issues every launch): the median of three runs
        out[name + "_fwd_bwd_ms"] = float(np.median([_device_ms(fwd_bwd, stream) for _ in range(3)]))
        out[name + "_psnr_db"] = float(np.mean(10 * np.log10(1.0 / mse)))
    out["time_ratio_full_over_sketched"] = out["full_fwd_bwd_ms"] / out["sketched_fwd_bwd_ms"]
    return out


# ---------------------------------------------------------------- native arm
def run_native(args, rank, world):
    import torch
    import paper_2203_07308_gb300 as pnp
    from paper_2203_07308_gb300 import build, synth

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    build.build()
    pnp.load()
    wl = workload(args.workload)
    if args.stage_iters is not None:
        wl = dataclasses.replace(wl, stages=[dataclasses.replace(s_, iters=min(s_.iters, args.stage_iters))
                                             for s_ in wl.stages])
    g = wl.geom
    B = g.batch
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    plan = pnp.Plan(g)

    # ---- synthetic inputs: B phantoms (other seeds per rank), b = A x + sigma w (GPU forward)
    d_xt, d_b = _simulate(plan, wl, dev, seed_offset=rank)
    seq = synth.schedule_sequence(wl.stages, synth.subset_seed(wl.config_id))
    total_iters = sum(s.iters for s in wl.stages)

    # ---- per-geometry set-up (not part of a step): step sizes eta_k = 1/L_k computed
    # by the library, and the launch shapes chosen by its autotuner for this schedule
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    eta = plan.step_sizes(wl.stages) if args.eta is None else [args.eta] * len(wl.stages)
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
    d_x = torch.zeros(B, g.n, g.n, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def step():
        plan.run(wl.stages, eta, seq, d_b, d_x.zero_(), graph=use_graph, **kw)

    launches_setup = pnp.launch_count()
    warm = args.warmup if args.profile else max(args.warmup, 3)
    for _ in range(warm):
        step()
    torch.cuda.synchronize()
    barrier(world)

    if args.profile:
        launches_warm = pnp.launch_count()
        torch.cuda.nvtx.range_push("timed")
        for _ in range(args.steps):
            step()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        if rank == 0:
            print(json.dumps({"profile": True, "steps": args.steps, "warmup": warm,
                              "launch_shapes": plan.launch_shapes(), "launches_before_timed": launches_warm,
                              "launches_per_step": (pnp.launch_count() - launches_warm) // max(args.steps, 1)}))
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
            step()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        barrier(world)
    launches = pnp.launch_count() - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = allmax(sum(step_ms), world)
    value = world * B * total_iters * args.steps / (total_ms / 1000.0)
    clocks = clk.summary()

    # ---- the same K steps again with a CUDA event pair on the run's stream
    # around every phase launch: each kernel's live launch durations.  (The
    # events cost a few microseconds of front-end time each, so the step above
    # carries none.)
    pnp.kernel_times(reset=True)
    ev_ph = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
             for _ in range(args.steps)]
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.fill_(float(k))
        ev_ph[k][0].record(stream)
        plan.run(wl.stages, eta, seq, d_b, d_x.zero_(), kernel_times=True, **kw)
        ev_ph[k][1].record(stream)
    torch.cuda.synchronize()
    phases = pnp.kernel_times(reset=True)
    ms_with_events = float(np.mean([a.elapsed_time(b) for a, b in ev_ph]))
    ph_ms = {k: v[0] for k, v in phases.items()}
    ph_n = {k: v[1] for k, v in phases.items()}

    # ---- the same step in the other launch mode (graph replay vs direct), for comparison
    other = []
    for k in range(5):
        flush.fill_(3.0)
        ms_ = _device_ms(lambda: plan.run(wl.stages, eta, seq, d_b, d_x.zero_(), graph=not use_graph, **kw), stream)
        if k >= 2:
            other.append(ms_)
    other_ms = float(np.median(other))

    # ---- all-view operators at this size: projector pair and full gradient A^T(Ax - b)
    def timed(fn, reps=10):
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

    res = torch.empty(B, g.n_views, g.n_det, device=dev)
    img = torch.empty(B, g.n, g.n, device=dev)
    fwd_ms = timed(lambda: plan.project(1, d_xt, res, d_b))
    back_ms = timed(lambda: plan.backproject(1, res, img))
    grad_ms = timed(lambda: plan.full_grad(d_xt, d_b, img))
    samples_full = plan.sample_count(1) * B

    # ---- time-to-PSNR: sketched schedule vs full-gradient PnP-FISTA, same data
    full_arm = synth.full_gradient_arm(wl.stages)
    eta_full = plan.step_sizes(full_arm)
    log_s = plan.run(wl.stages, eta, seq, d_b, d_x.zero_(), xtrue=d_xt, **kw)
    log_f = plan.run(full_arm, eta_full, None, d_b, d_x.zero_(), xtrue=d_xt, **kw)
    target = float(log_f[-1].mean()) - 0.1
    tts_s, it_s = _time_to_target(plan, wl.stages, eta, seq, d_b, d_x, log_s, target, kw, stream)
    tts_f, it_f = _time_to_target(plan, full_arm, eta_full, None, d_b, d_x, log_f, target, kw, stream)

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
    e2e_value = world * B * total_iters * len(e2e_ms) / (e2e_total / 1000.0)

    # ---- rooflines of the projector pair; the dominant kernel heads the line
    onchip = onchip_peaks()
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    clock_mhz = clocks.get("sm_max_mhz") or 2070.0
    samples_step = step_samples(plan, wl, seq)
    pixel_iters_step = float(B) * g.n * g.n * wl.tv_iters * total_iters
    per_kernel, alu_peak = rooflines(samples_step, pixel_iters_step, args.steps, ph_ms, ph_n, n_sm, clock_mhz, onchip)
    dominant = max(per_kernel, key=lambda k: ph_ms[k])
    dk = per_kernel[dominant]
    traffic = None
    kt = KERNEL_TRAFFIC.get(dominant)
    if kt and kt["bytes_per_unit"] and kt["sha256"] and kernel_source_sha(dominant) == kt["sha256"]:
        traffic = kt["bytes_per_unit"]
    work = (f"{FLOP_PER_PIXEL_ITER} FLOP per pixel and FGP iteration" if dominant == "denoise"
            else f"{FLOP_PER_SAMPLE} FLOP per projected sample")
    roof = {"kernel": dk["kernel"], "bound": "alu", "achieved": dk["alu"]["achieved"], "peak": alu_peak,
            "unit": "TFLOP/s", "frac": dk["alu"]["frac"], "traffic": traffic,
            "traffic_unit": kt["unit"] if kt else None,
            "work": work, "samples_per_step": samples_step, "pixel_iterations_per_step": pixel_iters_step,
            "units_per_step": ph_n[dominant] // args.steps, "mean_unit_us": dk["mean_unit_us"],
            "timing": (f"CUDA event pair on the run's stream around each of the {ph_n[dominant]} "
                       f"{dominant} phases of the K timed steps, re-run with phase events"),
            "peak_source": (f"{n_sm} SMs x 128 FP32 lanes x 2 FLOP (FMA) x {clock_mhz:.0f} MHz "
                            "(derived from the unit counts and the sampled maximum SM clock)"),
            "hbm_gbs_measured_peak": None}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            roof["hbm_gbs_measured_peak"] = json.load(f).get("hbm_gbs")
    except (OSError, ValueError):
        pass

    extras = {}
    if not args.no_extras:
        extras = {"single_256": single_256(dev, stream, args), "mixed_64": mixed_64(dev, stream),
                  "differentiable_256x8": differentiable_256x8(dev, stream),
                  "paper_sparse_view": paper_sparse_view(dev, kw),
                  "gray_by_config": gray_by_config(dev, stream)}

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
            "rooflines_per_kernel": per_kernel,
            "onchip_bandwidth_gbs": onchip,
            "full_gradients_per_s": B / (grad_ms / 1000.0),
            "kernels_ms_all_views": {"forward": fwd_ms, "backproject": back_ms, "full_gradient": grad_ms},
            "gray_samples_per_s_all_views": {"forward": samples_full / (fwd_ms / 1000) / 1e9,
                                             "backproject": samples_full / (back_ms / 1000) / 1e9,
                                             "samples_per_projection": samples_full},
            "time_to_psnr": {"target_db": target, "full_final_db": float(log_f[-1].mean()),
                             "sketched_final_db": float(log_s[-1].mean()),
                             "sketched_ms": tts_s, "sketched_iters": it_s,
                             "full_ms": tts_f, "full_iters": it_f,
                             "speedup": (tts_f / tts_s) if (tts_s and tts_f) else None},
            **extras,
            "setup_ms_step_sizes": setup_ms,
            "setup_ms_autotune": tune_ms,
            "step_sizes": eta,
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
