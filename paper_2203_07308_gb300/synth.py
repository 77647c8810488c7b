"""Seeded synthetic inputs: phantoms, noise draws, angle-subset sequences, workload table.

This module holds no arithmetic of the reconstruction method itself (no
projector, no gradient, no denoiser).  It produces only the inputs that both
the CUDA path and the FP64 oracle consume, so the two sides see identical data:

* ellipse phantoms ``x_true`` (the paper's "phantom image with disks of various
  sizes", Sec. 3, replaced by seeded random ellipses; its head and chest images
  are not available);
* standard-normal draws ``w`` for the additive measurement noise of the model
  ``b = A x_true + w`` (Eq. 1); the caller scales them by ``sigma * max|A x_true|``;
* the angle-subset order used by the minibatch gradient (Algorithm 1, Option 2):
  one seeded Fisher-Yates permutation of the subset ids per epoch;
* the fan-beam geometry of each workload, including the flat-detector pitch that
  makes the detector span the fan through the image's circumscribed circle.

All draws come from numpy's PCG64 generator with the stated seeds.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict
from typing import List, Optional, Tuple

import numpy as np


@dataclass(frozen=True)
class Geometry:
    """Fan-beam geometry in fine-pixel units (pixel side 1, image centred at the origin).

    Mirrors the C struct ``pnp_geom`` of the library and the oracle's geometry
    record: source at ``dso * (cos b, sin b)``, flat detector centred at
    ``-ddo * (cos b, sin b)`` with axis ``(-sin b, cos b)``, view ``v`` at angle
    ``b = angle0 + angle_span * v / n_views``, bin ``j`` centred at
    ``(j - (n_det - 1) / 2) * det_pitch``, fixed ray step ``step``.
    """

    n: int
    n_views: int
    n_det: int
    batch: int = 1
    dso: float = 0.0
    ddo: float = 0.0
    det_pitch: float = 0.0
    angle0: float = 0.0
    angle_span: float = 2.0 * math.pi
    step: float = 0.5

    def astuple(self) -> Tuple:
        return (self.n, self.n_views, self.n_det, self.batch, self.dso, self.ddo,
                self.det_pitch, self.angle0, self.angle_span, self.step)


def flat_detector_pitch(n: int, n_det: int, dso: float, ddo: float) -> float:
    """Pitch (fine px, at the detector) so that ``n_det`` bins exactly cover the fan
    of rays from the source tangent to the circle of radius ``n / sqrt(2)``."""
    r = n / math.sqrt(2.0)
    if dso <= r:
        raise ValueError("source must lie outside the image's circumscribed circle")
    return 2.0 * (dso + ddo) * r / (math.sqrt(dso * dso - r * r) * n_det)


def make_geometry(n: int, n_views: int, n_det: int, batch: int = 1, *,
                  dso_ratio: float = 2.0, ddo_ratio: float = 2.0,
                  angle0: float = 0.0, angle_span: float = 2.0 * math.pi,
                  step: float = 0.5) -> Geometry:
    """Geometry with source/detector distances given as multiples of the image width."""
    dso = dso_ratio * n
    ddo = ddo_ratio * n
    return Geometry(n=n, n_views=n_views, n_det=n_det, batch=batch, dso=dso, ddo=ddo,
                    det_pitch=flat_detector_pitch(n, n_det, dso, ddo),
                    angle0=angle0, angle_span=angle_span, step=step)


@dataclass(frozen=True)
class Stage:
    """One stage of the multi-stage schedule (Algorithm 1): sketch factor ``s``
    (average pool ``s x s``, so ``m_k = d / s^2``), number of inner iterations
    ``N_k`` and number of interleaved angle subsets ``P`` (1 = Option 1)."""

    factor: int
    iters: int
    n_subsets: int = 1
    kind: int = 0          # sketch: 0 s x s average pool, 1 bicubic (Keys a = -1/2, widened by s)
    estimator: int = 0     # subset gradient estimate (P > 1): 0 vanilla minibatch, 1 SVRG, 2 SAGA


@dataclass
class Workload:
    name: str
    geom: Geometry
    n_ellipses: Tuple[int, int]          # inclusive range of ellipse counts
    noise_rel: float                     # sigma as a fraction of max |A x_true|
    stages: List[Stage] = field(default_factory=list)
    tv_lambda: float = 0.02
    tv_iters: int = 20
    alpha: float = 1.0
    momentum: bool = True                # convergent-FISTA a_i = (i-1)/(i+3)
    config_id: int = 0                   # enters the phantom seed


def workloads() -> dict:
    """The five synthetic workloads (sizes, views, bins, noise, schedules)."""
    w = {}
    w["c1_64"] = Workload(
        name="64x64, 90 views x 96 bins, 30 PnP-PGD iterations, full gradient",
        geom=make_geometry(64, 90, 96), n_ellipses=(10, 10), noise_rel=0.01,
        stages=[Stage(1, 30, 1)], momentum=False, config_id=0)
    w["c2_256"] = Workload(
        name="256x256, 360 views x 512 bins, 2x sketch (20 it) then full (80 it), 8 angle subsets",
        geom=make_geometry(256, 360, 512), n_ellipses=(15, 20), noise_rel=0.01,
        stages=[Stage(2, 20, 8), Stage(1, 80, 8)], config_id=1)
    w["c3_512x16"] = Workload(
        name="16 x 512x512, 720 views x 768 bins, 4x/2x/full sketch stages, 12 angle subsets",
        geom=make_geometry(512, 720, 768, batch=16), n_ellipses=(15, 20), noise_rel=0.005,
        stages=[Stage(4, 24, 12), Stage(2, 24, 12), Stage(1, 72, 12)], config_id=2)
    w["c4_256x8"] = Workload(
        name="differentiable: 8 x 256x256, 360 views x 512 bins, 10 unrolled sketched iterations",
        geom=make_geometry(256, 360, 512, batch=8), n_ellipses=(15, 20), noise_rel=0.01,
        stages=[Stage(2, 10, 1)], config_id=3)
    return w


def paper_workloads() -> dict:
    """The three fan-beam set-ups of the paper's Sec. 3 (256x256 images, 228 bins
    so that A has 20520 or 82080 rows), on a synthetic disk-and-ellipse phantom
    (the head and chest images are not available), with Poisson transmission
    noise of the stated I0 and the paper's two-stage sketch (m_1 = d/16, then
    m_2 = d/4, Option 1).  Stage lengths are not given in the paper."""
    stages = [Stage(4, 30, 1), Stage(2, 70, 1)]
    return {
        "sparse_view": (Workload(name="sparse-view: 90 views over [0, 360), I0 = 10^5.5",
                                 geom=make_geometry(256, 90, 228), n_ellipses=(15, 20), noise_rel=0.0,
                                 stages=stages, config_id=10), 10 ** 5.5),
        "low_dose": (Workload(name="low-dose: 360 views over [0, 360), I0 = 10^3.5",
                              geom=make_geometry(256, 360, 228), n_ellipses=(15, 20), noise_rel=0.0,
                              stages=stages, config_id=11), 10 ** 3.5),
        "limited_angle": (Workload(name="limited-angle: 90 views over [0, 180), I0 = 10^5.5",
                                   geom=make_geometry(256, 90, 228, angle_span=math.pi), n_ellipses=(15, 20),
                                   noise_rel=0.0, stages=stages, config_id=12), 10 ** 5.5),
    }


def poisson_transmission(line_integrals: np.ndarray, i0: float, seed: int, mu: float = 0.02):
    """Transmission data of Sec. 3: counts ~ Poisson(I0 exp(-mu * A x)) and their
    log, b = -log(counts / I0) / mu, with the counts as weighted-least-squares
    weights (counts below 1 are raised to 1 before the log).  ``mu`` converts
    the phantom's unit intensities and pixel-length line integrals into an
    attenuation, so that the counts stay in a realistic range.  Returns
    (b, w) as float64 arrays shaped like ``line_integrals``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    expected = i0 * np.exp(-mu * np.asarray(line_integrals, dtype=np.float64))
    counts = np.maximum(rng.poisson(expected).astype(np.float64), 1.0)
    b = -np.log(counts / i0) / mu
    w = counts * mu * mu
    return b, w


def mixed_classes(n_instances: int = 64, seed: int = 5308):
    """Uneven serving-style mix: each of ``n_instances`` images draws one of three
    size classes (128x128 / 180 views x 256 bins, 256x256 / 360 x 512,
    512x512 / 720 x 768) uniformly with a seeded generator.  Returns
    [(Workload of that class with batch = its count, instance ids)]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pick = rng.integers(0, 3, size=n_instances)
    sizes = [(128, 180, 256), (256, 360, 512), (512, 720, 768)]
    out = []
    for c, (n, nv, nd) in enumerate(sizes):
        ids = np.nonzero(pick == c)[0]
        if ids.size == 0:
            continue
        wl = Workload(name=f"{n}x{n}, {nv} views x {nd} bins, {ids.size} images",
                      geom=make_geometry(n, nv, nd, batch=int(ids.size)), n_ellipses=(15, 20),
                      noise_rel=0.01, stages=[Stage(2, 20, 8), Stage(1, 30, 8)], config_id=4 + c)
        out.append((wl, ids))
    return out


def full_gradient_arm(stages: List[Stage]) -> List[Stage]:
    """The unsketched comparison arm (PnP-FISTA with the true gradient, Option 1)
    with the same total iteration count as ``stages``."""
    return [Stage(1, sum(s.iters for s in stages), 1)]


def phantom_seed(config_id: int, instance: int) -> int:
    return 2203 + 1000 * config_id + instance


def ellipse_phantom(n: int, seed: int, n_ellipses: Tuple[int, int] = (15, 20)) -> np.ndarray:
    """Sum of random filled ellipses evaluated at pixel centres, clipped to [0, 1].

    Centres uniform in the disk of radius 0.35 n, semi-axes uniform in
    [0.05 n, 0.25 n], rotation uniform in [0, pi), intensity uniform in [0, 1].
    Returns float64 ``[n, n]`` indexed ``[iy, ix]``; pixel ``(ix, iy)`` has centre
    ``(ix - (n-1)/2, iy - (n-1)/2)``.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    lo, hi = n_ellipses
    count = int(rng.integers(lo, hi + 1))
    c = (np.arange(n) - 0.5 * (n - 1)).astype(np.float64)
    X, Y = np.meshgrid(c, c, indexing="xy")
    img = np.zeros((n, n), dtype=np.float64)
    for _ in range(count):
        rad = 0.35 * n * math.sqrt(rng.random())
        ang = 2.0 * math.pi * rng.random()
        cx, cy = rad * math.cos(ang), rad * math.sin(ang)
        a = rng.uniform(0.05 * n, 0.25 * n)
        b = rng.uniform(0.05 * n, 0.25 * n)
        th = rng.uniform(0.0, math.pi)
        val = rng.random()
        ct, st = math.cos(th), math.sin(th)
        xr = (X - cx) * ct + (Y - cy) * st
        yr = -(X - cx) * st + (Y - cy) * ct
        img[(xr / a) ** 2 + (yr / b) ** 2 <= 1.0] += val
    return np.clip(img, 0.0, 1.0)


def phantom_batch(wl: Workload, batch: Optional[int] = None) -> np.ndarray:
    """``[B, n, n]`` float64 phantoms for a workload, one seed per instance."""
    b = wl.geom.batch if batch is None else batch
    return np.stack([ellipse_phantom(wl.geom.n, phantom_seed(wl.config_id, i), wl.n_ellipses)
                     for i in range(b)])


def noise_draws(shape, seed: int) -> np.ndarray:
    """Standard-normal draws (float64) for the additive noise term ``w`` of Eq. 1."""
    return np.random.Generator(np.random.PCG64(seed)).standard_normal(shape)


def noise_seed(config_id: int) -> int:
    return 7_000_000 + 1000 * config_id


def subset_sequence(n_iters: int, n_subsets: int, seed: int) -> np.ndarray:
    """Subset id for each of ``n_iters`` iterations: one Fisher-Yates permutation of
    ``0..n_subsets-1`` per epoch (numpy's ``permutation``), concatenated."""
    if n_subsets <= 1:
        return np.zeros(n_iters, dtype=np.int32)
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    while len(out) < n_iters:
        out.extend(int(p) for p in rng.permutation(n_subsets))
    return np.asarray(out[:n_iters], dtype=np.int32)


def schedule_sequence(stages: List[Stage], seed: int) -> np.ndarray:
    """Concatenated per-iteration subset ids for a multi-stage schedule."""
    parts = [subset_sequence(s.iters, s.n_subsets, seed + 17 * k) for k, s in enumerate(stages)]
    return np.concatenate(parts).astype(np.int32) if parts else np.zeros(0, np.int32)


def subset_seed(config_id: int) -> int:
    return 7308 + config_id


def describe(wl: Workload) -> dict:
    d = asdict(wl)
    d["geom"] = asdict(wl.geom)
    return d
