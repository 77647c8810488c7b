"""FP64 CPU oracle of the PnP-MS2G hot path — TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The product library (``paper_2203_07308_gb300``)
never imports, links or calls it, and it imports nothing from the product.

The arithmetic lives in ``pnp_oracle.c`` (plain C99, double precision, a naive
ray march for A and a naive scatter for A^T); this module compiles it with gcc
into ``oracle/_lib/`` and exposes numpy-level wrappers.  Each wrapper cites the
part of the paper it follows.

Parity status per function (what pins it, see ``tests/test_oracle_pins.py``):
  project / backproject   pinned (Gaussian-blob and paraboloid closed forms,
                           axis-ray row sums, dense matrix built two ways,
                           adjoint identity)
  pool / unpool           pinned (closed forms, adjoint identity)
  grad                    pinned (finite differences, subset-mean identity)
  power_iter              pinned (dense eigenvalue)
  fgp                     pinned at convergence (1-D step closed form,
                           independent primal-dual solve) and at 20 iterations
                           (generic dense FISTA on the dual problem)
  pnp_run                 pinned for one and four iterations against a dense
                           restatement of Algorithm 1; longer trajectories rest
                           on those step identities
  subset_sequence         pinned (published SplitMix64 outputs; every epoch a
                           permutation; uniform over all P! orders; one stream
                           across stages)
  sample_count            pinned exactly (closed forms for an axis ray, with
                           samples on the box edge, and a diagonal ray; the
                           chord-interval count of every ray of a full geometry)
The mutation tests (tests/test_oracle_mutations.py) plant plausible mistakes (one
per entry of their table) in a copy of pnp_oracle.c and check that these pins
catch each one.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pnp_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "libpnp_oracle.so")
# The mutation tests point this at a deliberately broken build of pnp_oracle.c
# to show that the pins catch plausible mistakes.
_LIB_OVERRIDE = os.environ.get("PNP_ORACLE_LIB")
_lock = threading.Lock()
_lib = None


class OrcGeom(C.Structure):
    _fields_ = [("n", C.c_int), ("n_views", C.c_int), ("n_det", C.c_int), ("batch", C.c_int),
                ("dso", C.c_double), ("ddo", C.c_double), ("pitch", C.c_double),
                ("angle0", C.c_double), ("span", C.c_double), ("step", C.c_double)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP over the rays of the forward projector and
    over fixed view chunks of the backprojector)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            if _LIB_OVERRIDE:
                lib = C.CDLL(_LIB_OVERRIDE)
            else:
                build()
                lib = C.CDLL(_LIB)
            dp = C.POINTER(C.c_double)
            gp = C.POINTER(OrcGeom)
            ip = C.POINTER(C.c_int)
            lib.orc_ray.argtypes = [gp, C.c_int, C.c_int, dp]
            lib.orc_subset_views.argtypes = [gp, C.c_int, C.c_int]
            lib.orc_subset_views.restype = C.c_int
            lib.orc_project.argtypes = [gp, C.c_int, dp, dp, dp, C.c_int, C.c_int]
            lib.orc_backproject.argtypes = [gp, C.c_int, dp, dp, C.c_int, C.c_int]
            lib.orc_pool.argtypes = [C.c_int, C.c_int, dp, dp]
            lib.orc_unpool.argtypes = [C.c_int, C.c_int, dp, dp]
            lib.orc_grad.argtypes = [gp, C.c_int, dp, dp, dp, C.c_int, C.c_int]
            lib.orc_fgp.argtypes = [C.c_int, dp, C.c_double, C.c_int, dp]
            lib.orc_tv.argtypes = [C.c_int, dp]
            lib.orc_tv.restype = C.c_double
            lib.orc_power_iter.argtypes = [gp, C.c_int, C.c_int, C.c_double, ip]
            lib.orc_power_iter.restype = C.c_double
            lib.orc_psnr.argtypes = [C.c_long, dp, dp]
            lib.orc_psnr.restype = C.c_double
            lib.orc_pnp_run.argtypes = [gp, C.c_int, ip, dp, ip, dp, dp, C.c_double, C.c_double,
                                        C.c_int, C.c_int, dp, dp]
            lib.orc_objective.argtypes = [gp, dp, dp, dp]
            lib.orc_grad_w.argtypes = [gp, C.c_int, dp, dp, dp, dp, C.c_int, C.c_int]
            lib.orc_grad_wk.argtypes = [gp, C.c_int, C.c_int, dp, dp, dp, dp, C.c_int, C.c_int]
            lib.orc_set_threads.argtypes = [C.c_int]
            lib.orc_get_threads.restype = C.c_int
            lib.orc_svrg_estimate.argtypes = [gp, C.c_int, C.c_int, dp, dp, dp, dp, dp, C.c_int, C.c_int, dp]
            lib.orc_saga_estimate.argtypes = [gp, C.c_int, C.c_int, dp, dp, dp, dp, C.c_int, C.c_int, dp]
            lib.orc_power_iter_wk.argtypes = [gp, C.c_int, C.c_int, dp, C.c_int, C.c_double, ip]
            lib.orc_power_iter_wk.restype = C.c_double
            lib.orc_keys.argtypes = [C.c_double]
            lib.orc_keys.restype = C.c_double
            lib.orc_splitmix64.argtypes = [C.c_uint64, C.c_uint64]
            lib.orc_splitmix64.restype = C.c_uint64
            lib.orc_subset_sequence.argtypes = [C.c_int, ip, C.c_uint64, ip]
            lib.orc_subset_sequence.restype = C.c_long
            lib.orc_bicubic_down.argtypes = [C.c_int, C.c_int, dp, dp]
            lib.orc_bicubic_up.argtypes = [C.c_int, C.c_int, dp, dp]
            lib.orc_power_iter_w.argtypes = [gp, C.c_int, dp, C.c_int, C.c_double, ip]
            lib.orc_power_iter_w.restype = C.c_double
            lib.orc_pnp_run_w.argtypes = [gp, C.c_int, ip, dp, ip, dp, dp, dp, C.c_double, C.c_double,
                                          C.c_int, C.c_int, dp, dp]
            lib.orc_objective_w.argtypes = [gp, dp, dp, dp, dp]
            lib.orc_fgp_vjp.argtypes = [C.c_int, dp, C.c_double, C.c_int, dp, dp, dp]
            lib.orc_step.argtypes = [gp, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                                     C.c_int, C.c_double, dp, dp, dp, dp, dp]
            lib.orc_step_vjp.argtypes = [gp, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                                         C.c_double, C.c_int, C.c_double, dp, dp, dp, dp, dp, dp, dp]
            lib.orc_sample_count.argtypes = [gp, C.c_int, C.c_int, C.c_int]
            lib.orc_sample_count.restype = C.c_double
            _lib = lib
    return _lib


def _dp(a: Optional[np.ndarray]):
    if a is None:
        return C.POINTER(C.c_double)()
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def geom(g) -> OrcGeom:
    """Oracle geometry record from any object with the ``pnp_geom`` field names."""
    return OrcGeom(int(g.n), int(g.n_views), int(g.n_det), int(getattr(g, "batch", 1)),
                   float(g.dso), float(g.ddo), float(g.det_pitch), float(g.angle0),
                   float(g.angle_span), float(g.step))


def ray(g, v: int, j: int) -> np.ndarray:
    """(S_x, S_y, d_x, d_y, F_x, F_y): source, unit direction and foot point of ray (v, j)."""
    out = np.zeros(6)
    _load().orc_ray(C.byref(geom(g)), v, j, _dp(out))
    return out


def subset_views(g, p: int, P: int) -> int:
    return _load().orc_subset_views(C.byref(geom(g)), p, P)


def project(g, s: int, img, b=None, p: int = 0, P: int = 1) -> np.ndarray:
    """A_s^{(p)} img (minus b^{(p)} if given); Eq. 1 / Eq. 4, Alg. 1 Option 2 rows."""
    lib = _load()
    gg = geom(g)
    img = _f64(img)
    nsub = lib.orc_subset_views(C.byref(gg), p, P)
    out = np.zeros((nsub, g.n_det))
    bb = None if b is None else _f64(b)
    lib.orc_project(C.byref(gg), s, _dp(img), _dp(bb), _dp(out), p, P)
    return out


def backproject(g, s: int, sino, p: int = 0, P: int = 1) -> np.ndarray:
    """A_s^{(p)T} sino by scatter (transpose of ``project``)."""
    ns = g.n // s
    out = np.zeros((ns, ns))
    sino = _f64(sino)
    _load().orc_backproject(C.byref(geom(g)), s, _dp(sino), _dp(out), p, P)
    return out


def pool(fine, s: int) -> np.ndarray:
    """Sketch S: s x s average pooling (Eq. 4's S, read as average pooling)."""
    fine = _f64(fine)
    n = fine.shape[-1]
    out = np.zeros((n // s, n // s))
    _load().orc_pool(n, s, _dp(fine), _dp(out))
    return out


def unpool(coarse, s: int) -> np.ndarray:
    """Upsampler U = S^T (replicate / s^2)."""
    coarse = _f64(coarse)
    n = coarse.shape[-1] * s
    out = np.zeros((n, n))
    _load().orc_unpool(n, s, _dp(coarse), _dp(out))
    return out


def keys(t: float) -> float:
    """Keys cubic convolution kernel, a = -1/2."""
    return float(_load().orc_keys(float(t)))


def bicubic_down(fine, s: int) -> np.ndarray:
    """Bicubic sketch S (separable Keys kernel widened by s, normalised)."""
    fine = _f64(fine)
    n = fine.shape[-1]
    out = np.zeros((n // s, n // s))
    _load().orc_bicubic_down(n, s, _dp(fine), _dp(out))
    return out


def bicubic_up(coarse, s: int) -> np.ndarray:
    """U = S^T of the bicubic sketch."""
    coarse = _f64(coarse)
    n = coarse.shape[-1] * s
    out = np.zeros((n, n))
    _load().orc_bicubic_up(n, s, _dp(coarse), _dp(out))
    return out


def grad(g, s: int, y, b, p: int = 0, P: int = 1, w=None, kind: int = 0) -> np.ndarray:
    """c S^T A_s^{(p)T} W^{(p)}(A_s^{(p)} S y - b^{(p)}), c = max(P, 1) (Alg. 1 G, U = S^T);
    W = diag(w) (weighted least squares) when w is given, else the identity."""
    y = _f64(y)
    b = _f64(b)
    ww = None if w is None else _f64(w)
    out = np.zeros((g.n, g.n))
    _load().orc_grad_wk(C.byref(geom(g)), s, int(kind), _dp(y), _dp(b), _dp(ww), _dp(out), p, P)
    return out


def fgp(z, lam: float, iters: int) -> np.ndarray:
    """TV-prox denoiser by FGP (Beck & Teboulle 2009), ``iters`` iterations."""
    z = _f64(z)
    out = np.zeros_like(z)
    _load().orc_fgp(z.shape[-1], _dp(z), float(lam), int(iters), _dp(out))
    return out


def tv(x) -> float:
    x = _f64(x)
    return float(_load().orc_tv(x.shape[-1], _dp(x)))


def power_iter(g, s: int, max_iters: int = 100, tol: float = 1e-7, w=None, kind: int = 0):
    """(L, iterations): L = ||W^{1/2} A_s S||^2 by power iteration (Sec. 3's eta = O(1/L))."""
    it = C.c_int(0)
    ww = None if w is None else _f64(w)
    L = _load().orc_power_iter_wk(C.byref(geom(g)), s, int(kind), _dp(ww), max_iters, tol, C.byref(it))
    return float(L), int(it.value)


def psnr(x, xt) -> float:
    x = _f64(x)
    xt = _f64(xt)
    return float(_load().orc_psnr(x.size, _dp(x), _dp(xt)))


def _stage_ints(stages) -> np.ndarray:
    """Stages as 5 ints each: factor, iters, n_subsets, kind, estimator."""
    return np.ascontiguousarray(np.array([[s.factor, s.iters, s.n_subsets, getattr(s, "kind", 0),
                                           getattr(s, "estimator", 0)]
                                          if hasattr(s, "factor") else (list(s) + [0, 0])[:5]
                                          for s in stages], dtype=np.int32).ravel())


def splitmix64(seed: int, t: int) -> int:
    """The t-th number (t >= 1) of the SplitMix64 stream with this seed
    (Steele, Lea & Flood 2014), the generator of the subset order."""
    return int(_load().orc_splitmix64(seed & (2**64 - 1), t))


def subset_sequence(stages: Sequence, seed: int) -> np.ndarray:
    """Subset id of every iteration of Algorithm 1's schedule: per stage with
    P > 1 subsets, one uniform permutation of the subsets per epoch of P
    iterations (Fisher-Yates on a seeded SplitMix64 stream); zeros for P = 1.
    The minibatch of each iteration is drawn at random (Sec. 2, Eq. 6-7)."""
    st = _stage_ints(stages)
    out = np.zeros(max(int(sum(st[1::5])), 1), np.int32)
    n = _load().orc_subset_sequence(len(st) // 5, st.ctypes.data_as(C.POINTER(C.c_int)),
                                    seed & (2**64 - 1), out.ctypes.data_as(C.POINTER(C.c_int)))
    return out[:n]


def pnp_run(g, stages: Sequence, eta: Sequence[float], seq, b, x0=None, *, alpha: float = 1.0,
            lam: float = 0.02, tv_iters: int = 20, momentum: bool = True, xt=None, w=None):
    """Algorithm 1 on one image; returns (x, psnr_log or None)."""
    st = _stage_ints(stages)
    total = int(sum(st[1::5]))
    seq = np.ascontiguousarray(np.asarray(seq, dtype=np.int32))
    if seq.size < total:
        seq = np.concatenate([seq, np.zeros(total - seq.size, np.int32)])
    eta = _f64(eta)
    b = _f64(b)
    x = np.zeros((g.n, g.n)) if x0 is None else _f64(x0).copy()
    xt_ = None if xt is None else _f64(xt)
    log = np.zeros(total) if xt is not None else None
    ip = C.POINTER(C.c_int)
    ww = None if w is None else _f64(w)
    _load().orc_pnp_run_w(C.byref(geom(g)), len(st) // 5, st.ctypes.data_as(ip), _dp(eta),
                          seq.ctypes.data_as(ip), _dp(b), _dp(ww), _dp(x), float(alpha), float(lam),
                          int(tv_iters), int(bool(momentum)), _dp(xt_), _dp(log))
    return x, log


def svrg_estimate(g, s: int, y, yt, mu, b, p: int, P: int, w=None, kind: int = 0) -> np.ndarray:
    """SVRG estimate G_p(y) - G_p(yt) + mu (Johnson & Zhang 2013), G_p the vanilla
    subset estimate of grad() (scaled by P); mu the full sketched gradient at yt."""
    out = np.zeros((g.n, g.n))
    ww = None if w is None else _f64(w)
    _load().orc_svrg_estimate(C.byref(geom(g)), s, int(kind), _dp(_f64(y)), _dp(_f64(yt)), _dp(_f64(mu)),
                              _dp(_f64(b)), _dp(ww), p, P, _dp(out))
    return out


def saga_estimate(g, s: int, y, psi, b, p: int, P: int, w=None, kind: int = 0) -> np.ndarray:
    """SAGA estimate G_p(y) - psi_p + mean_j psi_j (Defazio et al. 2014); updates
    psi[p] = G_p(y) in place (psi: float64 array [P, n, n])."""
    assert psi.dtype == np.float64 and psi.flags.c_contiguous and psi.shape == (P, g.n, g.n)
    out = np.zeros((g.n, g.n))
    ww = None if w is None else _f64(w)
    _load().orc_saga_estimate(C.byref(geom(g)), s, int(kind), _dp(_f64(y)), _dp(psi), _dp(_f64(b)), _dp(ww),
                              p, P, _dp(out))
    return out


def set_threads(n: int) -> int:
    """Sets the OpenMP thread count of the oracle's parallel loops (timing only);
    returns the previous count."""
    lib = _load()
    old = int(lib.orc_get_threads())
    lib.orc_set_threads(int(n))
    return old


def objective(g, x, b, w=None):
    """(1/2 sum_j w_j (A x - b)_j^2, TV(x)); w = 1 when not given."""
    out = np.zeros(2)
    x = _f64(x)
    b = _f64(b)
    ww = None if w is None else _f64(w)
    _load().orc_objective_w(C.byref(geom(g)), _dp(x), _dp(b), _dp(ww), _dp(out))
    return float(out[0]), float(out[1])


def sample_count(g, s: int = 1, p: int = 0, P: int = 1) -> float:
    """Exact number of samples inside the support box over the subset's rays."""
    return float(_load().orc_sample_count(C.byref(geom(g)), s, p, P))


def simulate(g, x_true, w, noise_rel: float):
    """b = A x_true + sigma w with sigma = noise_rel * max|A x_true| (Eq. 1)."""
    ax = project(g, 1, x_true)
    return ax + noise_rel * np.abs(ax).max() * _f64(w).reshape(ax.shape)


# ---------------------------------------------------------------- differentiable form
def fgp_vjp(z, lam: float, iters: int, xbar):
    """(zbar, lambar): reverse-mode derivative of ``fgp`` (Beck & Teboulle's FGP
    unrolled for ``iters`` iterations) applied to the output gradient ``xbar``."""
    z = _f64(z)
    xbar = _f64(xbar)
    zbar = np.zeros_like(z)
    lb = C.c_double(0.0)
    _load().orc_fgp_vjp(z.shape[-1], _dp(z), float(lam), int(iters), _dp(xbar), _dp(zbar), C.byref(lb))
    return zbar, float(lb.value)


def step(g, s: int, p: int, P: int, eta: float, alpha: float, lam: float, tv_iters: int, amom: float,
         y, xprev, b):
    """One iteration of Algorithm 1: returns (x_i, y_i) from (y_{i-1}, x_{i-1})."""
    y = _f64(y)
    xprev = _f64(xprev)
    b = _f64(b)
    xo = np.zeros_like(y)
    yo = np.zeros_like(y)
    _load().orc_step(C.byref(geom(g)), s, p, P, eta, alpha, lam, tv_iters, amom, _dp(y), _dp(xprev),
                     _dp(b), _dp(xo), _dp(yo))
    return xo, yo


def step_vjp(g, s: int, p: int, P: int, eta: float, alpha: float, lam: float, tv_iters: int,
             amom: float, y, b, xbar, ybar):
    """VJP of ``step``: (dJ/dy_{i-1}, dJ/dx_{i-1}, dJ/dlambda)."""
    y = _f64(y)
    b = _f64(b)
    xbar = _f64(xbar)
    ybar = _f64(ybar)
    yb = np.zeros_like(y)
    xpb = np.zeros_like(y)
    lb = C.c_double(0.0)
    _load().orc_step_vjp(C.byref(geom(g)), s, p, P, eta, alpha, lam, tv_iters, amom, _dp(y), _dp(b),
                         _dp(xbar), _dp(ybar), _dp(yb), _dp(xpb), C.byref(lb))
    return yb, xpb, float(lb.value)
