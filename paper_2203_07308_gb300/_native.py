"""ctypes binding of libpnp_ms2g.so (C ABI in include/pnp_ms2g.h).

Argument marshalling only: every numerical step runs in the library's CUDA
kernels.  Tensors are PyTorch CUDA tensors (device memory and streams come from
PyTorch); they are checked for device, dtype, contiguity and size, and passed
as raw pointers.  There is no fallback: if the library is missing or a call
fails, a ``PnpError`` is raised.
"""
from __future__ import annotations

import ctypes as C
import os
import re
import threading
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libpnp_ms2g.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "pnp_ms2g.h")

PNP_OK, PNP_EINVAL, PNP_ECUDA, PNP_ETIMEOUT, PNP_EUNSUPPORTED, PNP_ESTATE = range(6)
MAX_LOG_ITERS = 65536
NOALLOC_SCRATCH_BYTES = 32 << 20


class PnpError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"pnp error {code}: {msg}")
        self.code = code


class Geom(C.Structure):
    _fields_ = [("n", C.c_int32), ("n_views", C.c_int32), ("n_det", C.c_int32), ("batch", C.c_int32),
                ("dso", C.c_double), ("ddo", C.c_double), ("det_pitch", C.c_double),
                ("angle0", C.c_double), ("angle_span", C.c_double), ("step", C.c_double)]


class StageC(C.Structure):
    _fields_ = [("factor", C.c_int32), ("iters", C.c_int32), ("n_subsets", C.c_int32), ("kind", C.c_int32),
                ("estimator", C.c_int32)]


class LaunchShapes(C.Structure):
    _fields_ = [("lanes", C.c_int32 * 4), ("back", C.c_int32 * 4), ("tile", C.c_int32)]


BACK_TILE4 = 1 << 8     # backprojector CTAs of 4 x 4 pixel blocks (| view groups)
BACK_SCATTER = 1 << 9   # backprojector as the fixed-point scatter (| tile side 12, 16, 22 or 32)
BACK_TABLE = 1 << 10    # backprojector reading the stored gather table (| BACK_BATCH(bc) | view groups)


def BACK_BATCH(bc):
    """Images per thread of the batched and table gathers (PNP_BACK_BATCH)."""
    return int(bc) << 16

SKETCH_POOL, SKETCH_BICUBIC = 0, 1
EST_MINIBATCH, EST_SVRG, EST_SAGA = 0, 1, 2


class RunParams(C.Structure):
    _fields_ = [("alpha", C.c_float), ("lambda_", C.c_float), ("tv_iters", C.c_int32),
                ("momentum", C.c_int32), ("flags", C.c_int32), ("subset_seed", C.c_uint64)]


RUN_GRAPH = 1
RUN_KERNEL_TIMES = 2
RUN_PERSISTENT = 4     # phase kernels in their persistent form (CTAs that fit at once walk the work table)
PHASES = ("prep", "forward", "backward", "denoise")


class ProblemC(C.Structure):
    _fields_ = [("geom", Geom), ("stages", C.POINTER(StageC)), ("n_stages", C.c_int32),
                ("h_eta", C.POINTER(C.c_double)), ("h_subset_seq", C.POINTER(C.c_int32)),
                ("d_b", C.c_void_p), ("d_x", C.c_void_p), ("d_xtrue", C.c_void_p),
                ("h_psnr_log", C.POINTER(C.c_double)), ("d_ws", C.c_void_p),
                ("start_iter", C.c_int32), ("d_y", C.c_void_p)]


_lock = threading.Lock()
_lib = None


def header_functions() -> list:
    """Names of the functions that include/pnp_ms2g.h declares."""
    with open(HEADER) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pnp_[a-z0-9_]+)\s*\(", text)))


def load(path: Optional[str] = None):
    """Load the library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise PnpError(PNP_EUNSUPPORTED,
                           f"{p} not built: run `python -m paper_2203_07308_gb300.build`")
        lib = C.CDLL(p)
        vp, i32, sz = C.c_void_p, C.c_int, C.c_size_t
        gp = C.POINTER(Geom)
        dp = C.POINTER(C.c_double)
        sig = {
            "pnp_workspace_size": [gp, C.POINTER(sz)],
            "pnp_setup": [gp, vp, sz, vp],
            "pnp_project": [gp, i32, vp, vp, vp, i32, i32, vp, vp],
            "pnp_backproject": [gp, i32, vp, vp, i32, i32, vp, vp],
            "pnp_sketch": [gp, i32, vp, vp, vp],
            "pnp_upsample": [gp, i32, vp, vp, vp],
            "pnp_full_grad": [gp, vp, vp, vp, vp, vp],
            "pnp_sketch_grad": [gp, i32, vp, vp, vp, i32, i32, vp, vp],
            "pnp_tv_workspace_size": [i32, i32, C.POINTER(sz)],
            "pnp_tv_denoise": [vp, vp, i32, i32, C.c_float, i32, vp, sz, vp],
            "pnp_power_iter": [gp, i32, i32, C.c_double, dp, C.POINTER(i32), vp, vp],
            "pnp_run": [gp, C.POINTER(StageC), i32, dp, C.POINTER(C.c_int32), C.POINTER(RunParams),
                        vp, vp, vp, dp, vp, vp],
            "pnp_objective": [gp, vp, vp, vp, dp, vp, vp],
            "pnp_sample_count": [gp, i32, i32, i32, dp, vp, vp],
            "pnp_full_grad_noalloc": [gp, vp, vp, vp, vp],
            "pnp_run_many": [C.POINTER(ProblemC), i32, C.POINTER(RunParams), vp],
            "pnp_set_weights": [gp, vp, vp],
            "pnp_sketch_kind": [gp, i32, i32, vp, vp, vp],
            "pnp_kernel_times": [dp, C.POINTER(C.c_int64), i32],
            "pnp_vr_buffer_size": [gp, C.POINTER(StageC), i32, C.POINTER(sz)],
            "pnp_get_launch_shapes": [gp, C.POINTER(LaunchShapes), vp],
            "pnp_set_launch_shapes": [gp, C.POINTER(LaunchShapes), vp],
            "pnp_set_vr_buffer": [gp, vp, sz, vp],
            "pnp_gather_table_size": [gp, vp, C.POINTER(sz), vp],
            "pnp_set_gather_table": [gp, vp, sz, vp, vp],
            "pnp_upsample_kind": [gp, i32, i32, vp, vp, vp],
            "pnp_sketch_grad_kind": [gp, i32, i32, vp, vp, vp, i32, i32, vp, vp],
            "pnp_power_iter_kind": [gp, i32, i32, i32, C.c_double, dp, C.POINTER(i32), vp, vp],
            "pnp_autotune": [gp, C.POINTER(StageC), i32, C.POINTER(RunParams), vp, vp],
            "pnp_tv_vjp_workspace_size": [i32, i32, i32, C.POINTER(sz)],
            "pnp_tv_vjp": [vp, vp, vp, dp, i32, i32, C.c_float, i32, vp, sz, vp],
            "pnp_vjp_workspace_size": [gp, i32, C.POINTER(sz)],
            "pnp_unrolled_step": [gp, i32, i32, i32, C.c_double, C.POINTER(RunParams), C.c_float,
                                  vp, vp, vp, vp, vp, vp, vp],
            "pnp_unrolled_step_vjp": [gp, i32, i32, i32, C.c_double, C.POINTER(RunParams), C.c_float,
                                      vp, vp, vp, vp, vp, vp, dp, vp, vp, sz, vp],
            "pnp_unrolled_step_save": [gp, i32, i32, i32, C.c_double, C.POINTER(RunParams), C.c_float,
                                       vp, vp, vp, vp, vp, vp, vp, vp],
            "pnp_unrolled_step_vjp_saved": [gp, i32, i32, i32, C.c_double, C.POINTER(RunParams), C.c_float,
                                            vp, vp, vp, vp, vp, dp, vp, vp, sz, vp],
            "pnp_step_sizes": [gp, C.POINTER(StageC), i32, dp, vp, vp],
            "pnp_schedule": [C.POINTER(StageC), i32, C.POINTER(C.c_int32), i32, C.POINTER(C.c_int32),
                             C.POINTER(C.c_int32), C.POINTER(C.c_float), C.c_int64, C.POINTER(C.c_int64)],
            "pnp_subset_sequence": [C.POINTER(StageC), i32, C.c_uint64, C.POINTER(C.c_int32), C.c_int64,
                                    C.POINTER(C.c_int64)],
            "pnp_onchip_bandwidth": [vp, sz, dp, vp],
        }
        for name, args in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = C.c_int
        lib.pnp_launch_count.argtypes = []
        lib.pnp_launch_count.restype = C.c_uint64
        lib.pnp_last_error.argtypes = []
        lib.pnp_last_error.restype = C.c_char_p
        _lib = lib
        return lib


def _check(code: int):
    if code != PNP_OK:
        msg = load().pnp_last_error().decode(errors="replace")
        raise PnpError(code, msg)


def geom(g) -> Geom:
    """C geometry record from a ``synth.Geometry`` (or anything with its fields)."""
    if isinstance(g, Geom):
        return g
    return Geom(int(g.n), int(g.n_views), int(g.n_det), int(getattr(g, "batch", 1)), float(g.dso),
                float(g.ddo), float(g.det_pitch), float(g.angle0), float(g.angle_span), float(g.step))


def _stream(stream) -> C.c_void_p:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream))


def _ptr(t, numel: Optional[int] = None, name: str = "tensor", allow_none: bool = False):
    if t is None:
        if allow_none:
            return None
        raise PnpError(PNP_EINVAL, f"{name} is required")
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise PnpError(PNP_EINVAL, f"{name} must be a CUDA tensor")
    if t.dtype != torch.float32:
        raise PnpError(PNP_EINVAL, f"{name} must be float32")
    if not t.is_contiguous():
        raise PnpError(PNP_EINVAL, f"{name} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise PnpError(PNP_EINVAL, f"{name} has {t.numel()} elements, expected {numel}")
    return C.c_void_p(t.data_ptr())


def _ws(ws):
    import torch
    if not isinstance(ws, torch.Tensor) or not ws.is_cuda:
        raise PnpError(PNP_EINVAL, "workspace must be a CUDA tensor")
    return C.c_void_p(ws.data_ptr()), ws.numel() * ws.element_size()


def subset_views(g, p: int, P: int) -> int:
    return g.n_views if P <= 1 else (g.n_views - p + P - 1) // P


# ---------------------------------------------------------------- entry points
def workspace_size(g) -> int:
    n = C.c_size_t(0)
    _check(load().pnp_workspace_size(C.byref(geom(g)), C.byref(n)))
    return int(n.value)


def setup(g, ws, stream=None):
    p, nbytes = _ws(ws)
    _check(load().pnp_setup(C.byref(geom(g)), p, nbytes, _stream(stream)))


def project(g, factor, img, sino, b=None, subset=0, n_subsets=1, ws=None, stream=None):
    ns = g.n // factor
    nsub = subset_views(g, subset, n_subsets)
    _check(load().pnp_project(C.byref(geom(g)), factor, _ptr(img, g.batch * ns * ns, "img"),
                              _ptr(b, g.batch * g.n_views * g.n_det, "b", True),
                              _ptr(sino, g.batch * nsub * g.n_det, "sino"), subset, n_subsets,
                              _ws(ws)[0], _stream(stream)))


def backproject(g, factor, sino, img, subset=0, n_subsets=1, ws=None, stream=None):
    ns = g.n // factor
    nsub = subset_views(g, subset, n_subsets)
    _check(load().pnp_backproject(C.byref(geom(g)), factor, _ptr(sino, g.batch * nsub * g.n_det, "sino"),
                                  _ptr(img, g.batch * ns * ns, "img"), subset, n_subsets,
                                  _ws(ws)[0], _stream(stream)))


def sketch(g, factor, fine, coarse, stream=None, kind=0):
    ns = g.n // factor
    _check(load().pnp_sketch_kind(C.byref(geom(g)), factor, int(kind), _ptr(fine, g.batch * g.n * g.n, "fine"),
                                  _ptr(coarse, g.batch * ns * ns, "coarse"), _stream(stream)))


def upsample(g, factor, coarse, fine, stream=None, kind=0):
    ns = g.n // factor
    _check(load().pnp_upsample_kind(C.byref(geom(g)), factor, int(kind), _ptr(coarse, g.batch * ns * ns, "coarse"),
                                    _ptr(fine, g.batch * g.n * g.n, "fine"), _stream(stream)))


def full_grad(g, x, b, out, ws, stream=None):
    img = g.batch * g.n * g.n
    _check(load().pnp_full_grad(C.byref(geom(g)), _ptr(x, img, "x"), _ptr(b, g.batch * g.n_views * g.n_det, "b"),
                                _ptr(out, img, "g"), _ws(ws)[0], _stream(stream)))


def full_grad_noalloc(g, x, b, out, stream=None):
    """pnp_full_grad_noalloc: the full gradient without a workspace (scratch inside
    the library, PNP_NOALLOC_SCRATCH_BYTES per GPU)."""
    img = g.batch * g.n * g.n
    _check(load().pnp_full_grad_noalloc(C.byref(geom(g)), _ptr(x, img, "x"),
                                        _ptr(b, g.batch * g.n_views * g.n_det, "b"), _ptr(out, img, "g"),
                                        _stream(stream)))


def sketch_grad(g, factor, y, b, out, subset=0, n_subsets=1, ws=None, stream=None, kind=0):
    img = g.batch * g.n * g.n
    _check(load().pnp_sketch_grad_kind(C.byref(geom(g)), factor, int(kind), _ptr(y, img, "y"),
                                       _ptr(b, g.batch * g.n_views * g.n_det, "b"), _ptr(out, img, "g"),
                                       subset, n_subsets, _ws(ws)[0], _stream(stream)))


def tv_workspace_size(n: int, batch: int) -> int:
    v = C.c_size_t(0)
    _check(load().pnp_tv_workspace_size(n, batch, C.byref(v)))
    return int(v.value)


def tv_denoise(z, x, n, batch, lam, iters, ws, stream=None):
    p, nbytes = _ws(ws) if ws is not None else (None, 0)
    _check(load().pnp_tv_denoise(_ptr(z, batch * n * n, "z"), _ptr(x, batch * n * n, "x"), n, batch,
                                 float(lam), int(iters), p, nbytes, _stream(stream)))


def power_iter(g, factor, max_iters=100, tol=1e-7, ws=None, stream=None, kind=0):
    L = C.c_double(0.0)
    it = C.c_int(0)
    _check(load().pnp_power_iter_kind(C.byref(geom(g)), factor, int(kind), max_iters, tol, C.byref(L),
                                      C.byref(it), _ws(ws)[0], _stream(stream)))
    return float(L.value), int(it.value)


def _stages(stages: Sequence):
    arr = (StageC * len(stages))()
    for k, s in enumerate(stages):
        f, it, P, kind, est = ((s.factor, s.iters, s.n_subsets, getattr(s, "kind", 0), getattr(s, "estimator", 0))
                               if hasattr(s, "factor") else (tuple(s) + (0, 0))[:5])
        arr[k] = StageC(int(f), int(it), int(P), int(kind), int(est))
    return arr


def vr_buffer_size(g, stages) -> int:
    """Bytes of the SVRG/SAGA estimator buffer the schedule needs (0 if none)."""
    st = _stages(stages)
    v = C.c_size_t(0)
    _check(load().pnp_vr_buffer_size(C.byref(geom(g)), st, len(st), C.byref(v)))
    return int(v.value)


def step_sizes(g, stages, ws, stream=None) -> list:
    """pnp_step_sizes: eta_k = 1/L_k of every stage (power iteration in the
    library, cached per workspace)."""
    st = _stages(stages)
    out = (C.c_double * len(st))()
    _check(load().pnp_step_sizes(C.byref(geom(g)), st, len(st), out, _ws(ws)[0], _stream(stream)))
    return [float(v) for v in out]


def schedule(stages, seq=None, momentum=True):
    """pnp_schedule: (stage index, subset id, momentum coefficient a_i) of every
    iteration of the schedule, as int32 / int32 / float32 arrays."""
    st = _stages(stages)
    total = sum(a.iters for a in st)
    seq_np = None if seq is None else np.ascontiguousarray(np.asarray(seq, dtype=np.int32))
    if seq_np is not None and seq_np.size < total:
        raise PnpError(PNP_EINVAL, "subset sequence shorter than the schedule")
    stage = np.zeros(max(total, 1), dtype=np.int32)
    subset = np.zeros(max(total, 1), dtype=np.int32)
    amom = np.zeros(max(total, 1), dtype=np.float32)
    n = C.c_int64(0)
    _check(load().pnp_schedule(st, len(st), None if seq_np is None else seq_np.ctypes.data_as(C.POINTER(C.c_int32)),
                               int(bool(momentum)), stage.ctypes.data_as(C.POINTER(C.c_int32)),
                               subset.ctypes.data_as(C.POINTER(C.c_int32)), amom.ctypes.data_as(C.POINTER(C.c_float)),
                               stage.size, C.byref(n)))
    return stage[:n.value], subset[:n.value], amom[:n.value]


def subset_sequence(stages, seed=0):
    """pnp_subset_sequence: the subset id of every iteration, one Fisher-Yates
    permutation of the stage's subsets per epoch drawn from a SplitMix64 stream
    with this seed (zeros for stages without subsets); int32 array."""
    st = _stages(stages)
    out = np.zeros(max(sum(a.iters for a in st), 1), dtype=np.int32)
    n = C.c_int64(0)
    _check(load().pnp_subset_sequence(st, len(st), int(seed) & (2**64 - 1),
                                      out.ctypes.data_as(C.POINTER(C.c_int32)), out.size, C.byref(n)))
    return out[:n.value]


def _seq_ptr(seq, total):
    """The caller's subset sequence as an int32 array and pointer; (None, None)
    when there is none (the library then draws the seeded order)."""
    if seq is None:
        return None, None
    seq_np = np.ascontiguousarray(np.asarray(seq, dtype=np.int32))
    if seq_np.size < total:
        raise PnpError(PNP_EINVAL, "subset sequence shorter than the schedule")
    return seq_np, seq_np.ctypes.data_as(C.POINTER(C.c_int32))


def onchip_bandwidth(device="cuda", stream=None) -> dict:
    """pnp_onchip_bandwidth: measured L2, L1 and shared-memory read bandwidth (GB/s)."""
    import torch
    buf = torch.empty(32 << 20, dtype=torch.uint8, device=device)
    out = (C.c_double * 3)()
    _check(load().pnp_onchip_bandwidth(C.c_void_p(buf.data_ptr()), buf.numel(), out, _stream(stream)))
    return {"l2_gbs": float(out[0]), "l1_gbs": float(out[1]), "smem_gbs": float(out[2])}


def _flags(graph, kernel_times, persistent=False):
    return (RUN_GRAPH if graph else 0) | (RUN_KERNEL_TIMES if kernel_times else 0) | \
        (RUN_PERSISTENT if persistent else 0)


def run(g, stages, eta, seq, b, x, *, alpha=1.0, lam=0.02, tv_iters=20, momentum=True,
        xtrue=None, ws=None, stream=None, graph=False, kernel_times=False, persistent=False,
        subset_seed=0):
    """Algorithm 1; x holds x_0 on entry and the result on return.  eta: step
    size per stage, or None for eta_k = 1/L_k computed by the library.  seq: the
    subset id of every iteration, or None for the library's order drawn from
    subset_seed (subset_sequence).  Returns the
    PSNR log [total_iters, batch] when xtrue is given, else None.  graph=True
    captures the launch sequence once per distinct call and replays it;
    kernel_times=True brackets each phase launch with CUDA events (read them
    with kernel_times())."""
    st = _stages(stages)
    total = sum(a.iters for a in st)
    eta_a = None if eta is None else (C.c_double * len(st))(*[float(e) for e in eta])
    seq_np, seq_p = _seq_ptr(seq, total)
    prm = RunParams(float(alpha), float(lam), int(tv_iters), int(bool(momentum)),
                    _flags(graph, kernel_times, persistent), int(subset_seed) & (2**64 - 1))
    img = g.batch * g.n * g.n
    log = np.zeros((total, g.batch)) if xtrue is not None else None
    _check(load().pnp_run(C.byref(geom(g)), st, len(st), eta_a,
                          seq_p, C.byref(prm),
                          _ptr(b, g.batch * g.n_views * g.n_det, "b"), _ptr(x, img, "x"),
                          _ptr(xtrue, img, "xtrue", True),
                          log.ctypes.data_as(C.POINTER(C.c_double)) if log is not None else None,
                          _ws(ws)[0], _stream(stream)))
    return log


def objective(g, x, b, xtrue=None, ws=None, stream=None):
    out = np.zeros((g.batch, 3))
    img = g.batch * g.n * g.n
    _check(load().pnp_objective(C.byref(geom(g)), _ptr(x, img, "x"),
                                _ptr(b, g.batch * g.n_views * g.n_det, "b"),
                                _ptr(xtrue, img, "xtrue", True), out.ctypes.data_as(C.POINTER(C.c_double)),
                                _ws(ws)[0], _stream(stream)))
    return out


def sample_count(g, factor=1, subset=0, n_subsets=1, ws=None, stream=None) -> float:
    v = C.c_double(0.0)
    _check(load().pnp_sample_count(C.byref(geom(g)), factor, subset, n_subsets, C.byref(v),
                                   _ws(ws)[0], _stream(stream)))
    return float(v.value)


def kernel_times(reset=False):
    """{phase: (device ms summed, launches)} over runs made with kernel_times=True."""
    ms = (C.c_double * len(PHASES))()
    cnt = (C.c_int64 * len(PHASES))()
    _check(load().pnp_kernel_times(ms, cnt, int(bool(reset))))
    return {ph: (float(ms[k]), int(cnt[k])) for k, ph in enumerate(PHASES)}


def launch_count() -> int:
    return int(load().pnp_launch_count())


def last_error() -> str:
    return load().pnp_last_error().decode(errors="replace")


class Plan:
    """A geometry with its device workspace allocated (by PyTorch) and prepared."""

    def __init__(self, g, device="cuda", stream=None, gather_table=False):
        import torch
        self.g = g
        self.cg = geom(g)
        self.ws = torch.empty(workspace_size(g), dtype=torch.uint8, device=device)
        setup(g, self.ws, stream)
        self.table = None
        if gather_table:
            self.set_gather_table(stream=stream)

    def gather_table_size(self, stream=None) -> int:
        """Bytes of the stored gather table of this geometry (pnp_gather_table_size)."""
        n = C.c_size_t(0)
        _check(load().pnp_gather_table_size(C.byref(self.cg), _ws(self.ws)[0], C.byref(n), _stream(stream)))
        return int(n.value)

    def set_gather_table(self, enable=True, stream=None):
        """Allocates (PyTorch), builds and registers the stored gather table, or
        unregisters and frees it (enable=False)."""
        import torch
        if not enable:
            _check(load().pnp_set_gather_table(C.byref(self.cg), None, 0, _ws(self.ws)[0], _stream(stream)))
            self.table = None
            return
        n = self.gather_table_size(stream)
        buf = torch.empty(max(n, 256), dtype=torch.uint8, device=self.ws.device)
        _check(load().pnp_set_gather_table(C.byref(self.cg), C.c_void_p(buf.data_ptr()), buf.numel(),
                                           _ws(self.ws)[0], _stream(stream)))
        self.table = buf

    def project(self, factor, img, sino, b=None, subset=0, n_subsets=1, stream=None):
        project(self.g, factor, img, sino, b, subset, n_subsets, self.ws, stream)

    def backproject(self, factor, sino, img, subset=0, n_subsets=1, stream=None):
        backproject(self.g, factor, sino, img, subset, n_subsets, self.ws, stream)

    def full_grad(self, x, b, out, stream=None):
        full_grad(self.g, x, b, out, self.ws, stream)

    def sketch_grad(self, factor, y, b, out, subset=0, n_subsets=1, stream=None, kind=0):
        sketch_grad(self.g, factor, y, b, out, subset, n_subsets, self.ws, stream, kind)

    def power_iter(self, factor, max_iters=100, tol=1e-7, stream=None, kind=0):
        return power_iter(self.g, factor, max_iters, tol, self.ws, stream, kind)

    def step_sizes(self, stages, stream=None):
        return step_sizes(self.g, stages, self.ws, stream)

    def ensure_vr_buffer(self, stages):
        """Allocates (PyTorch) and registers the SVRG/SAGA state buffer the
        schedule needs, keeping a large enough one that is already registered."""
        import torch
        need = vr_buffer_size(self.g, stages)
        have = getattr(self, "vr", None)
        if need == 0 or (have is not None and have.numel() >= need):
            return
        self.set_vr_buffer(torch.empty(need, dtype=torch.uint8, device=self.ws.device))

    def set_vr_buffer(self, buf):
        self.vr = buf
        p, n = (None, 0) if buf is None else (C.c_void_p(buf.data_ptr()), buf.numel() * buf.element_size())
        _check(load().pnp_set_vr_buffer(C.byref(self.cg), p, n, _ws(self.ws)[0]))

    def run(self, stages, eta, seq, b, x, **kw):
        self.ensure_vr_buffer(stages)
        return run(self.g, stages, eta, seq, b, x, ws=self.ws, **kw)

    def autotune(self, stages, **kw):
        autotune(self.g, stages, self.ws, **kw)

    def launch_shapes(self) -> dict:
        """{"lanes": [4], "back": [4], "tile": int} of this workspace (0 = heuristic)."""
        ls = LaunchShapes()
        _check(load().pnp_get_launch_shapes(C.byref(self.cg), C.byref(ls), _ws(self.ws)[0]))
        return {"lanes": list(ls.lanes), "back": list(ls.back), "tile": int(ls.tile)}

    def set_launch_shapes(self, lanes=(0, 0, 0, 0), back=(0, 0, 0, 0), tile=0):
        """Pins launch shapes per level (factors 1, 2, 4, 8): forward lanes per ray,
        backprojector view groups, FGP tile side (0 = heuristic)."""
        ls = LaunchShapes((C.c_int32 * 4)(*lanes), (C.c_int32 * 4)(*back), int(tile))
        _check(load().pnp_set_launch_shapes(C.byref(self.cg), C.byref(ls), _ws(self.ws)[0]))

    def set_weights(self, w):
        """Weighted least squares for every gradient of this plan (None: unweighted)."""
        self.weights = w
        p = None if w is None else _ptr(w, self.g.batch * self.g.n_views * self.g.n_det, "w")
        _check(load().pnp_set_weights(C.byref(self.cg), p, _ws(self.ws)[0]))

    def objective(self, x, b, xtrue=None, stream=None):
        return objective(self.g, x, b, xtrue, self.ws, stream)

    def sample_count(self, factor=1, subset=0, n_subsets=1, stream=None):
        return sample_count(self.g, factor, subset, n_subsets, self.ws, stream)


# ---------------------------------------------------------------- differentiable form
def tv_vjp_workspace_size(n: int, batch: int, iters: int) -> int:
    v = C.c_size_t(0)
    _check(load().pnp_tv_vjp_workspace_size(n, batch, iters, C.byref(v)))
    return int(v.value)


def tv_vjp(z, xbar, zbar, n, batch, lam, iters, ws, stream=None):
    """pnp_tv_vjp: zbar = (dD/dz)^T xbar; returns dJ/dlambda per instance."""
    lb = np.zeros(batch)
    p, nbytes = _ws(ws) if ws is not None else (None, 0)
    img = batch * n * n
    _check(load().pnp_tv_vjp(_ptr(z, img, "z"), _ptr(xbar, img, "xbar"), _ptr(zbar, img, "zbar"),
                             lb.ctypes.data_as(C.POINTER(C.c_double)), n, batch, float(lam), int(iters),
                             p, nbytes, _stream(stream)))
    return lb


def vjp_workspace_size(g, tv_iters: int) -> int:
    v = C.c_size_t(0)
    _check(load().pnp_vjp_workspace_size(C.byref(geom(g)), int(tv_iters), C.byref(v)))
    return int(v.value)


def unrolled_step(g, factor, subset, n_subsets, eta, alpha, lam, tv_iters, amom, y, xprev, b, xout, yout,
                  ws, stream=None):
    img = g.batch * g.n * g.n
    prm = RunParams(float(alpha), float(lam), int(tv_iters), 0, 0)
    _check(load().pnp_unrolled_step(C.byref(geom(g)), factor, subset, n_subsets, float(eta), C.byref(prm),
                                    float(amom), _ptr(y, img, "y"), _ptr(xprev, img, "xprev"),
                                    _ptr(b, g.batch * g.n_views * g.n_det, "b"), _ptr(xout, img, "xout"),
                                    _ptr(yout, img, "yout"), _ws(ws)[0], _stream(stream)))


def unrolled_step_save(g, factor, subset, n_subsets, eta, alpha, lam, tv_iters, amom, y, xprev, b, xout, yout,
                       zout, ws, stream=None):
    """unrolled_step that also stores the gradient step z into zout."""
    img = g.batch * g.n * g.n
    prm = RunParams(float(alpha), float(lam), int(tv_iters), 0, 0)
    _check(load().pnp_unrolled_step_save(C.byref(geom(g)), factor, subset, n_subsets, float(eta), C.byref(prm),
                                         float(amom), _ptr(y, img, "y"), _ptr(xprev, img, "xprev"),
                                         _ptr(b, g.batch * g.n_views * g.n_det, "b"), _ptr(xout, img, "xout"),
                                         _ptr(yout, img, "yout"), _ptr(zout, img, "zout"), _ws(ws)[0],
                                         _stream(stream)))


def unrolled_step_vjp_saved(g, factor, subset, n_subsets, eta, alpha, lam, tv_iters, amom, z, xbar, ybar,
                            ybar_in, xpbar, ws, vjp_ws, stream=None):
    """unrolled_step_vjp from the stored z; returns dJ/dlambda per instance."""
    img = g.batch * g.n * g.n
    prm = RunParams(float(alpha), float(lam), int(tv_iters), 0, 0)
    lb = np.zeros(g.batch)
    vp, vbytes = _ws(vjp_ws)
    _check(load().pnp_unrolled_step_vjp_saved(C.byref(geom(g)), factor, subset, n_subsets, float(eta),
                                              C.byref(prm), float(amom), _ptr(z, img, "z"),
                                              _ptr(xbar, img, "xbar"), _ptr(ybar, img, "ybar"),
                                              _ptr(ybar_in, img, "ybar_in"), _ptr(xpbar, img, "xpbar"),
                                              lb.ctypes.data_as(C.POINTER(C.c_double)), _ws(ws)[0], vp, vbytes,
                                              _stream(stream)))
    return lb


def unrolled_step_vjp(g, factor, subset, n_subsets, eta, alpha, lam, tv_iters, amom, y, b, xbar, ybar,
                      ybar_in, xpbar, ws, vjp_ws, stream=None):
    """Returns dJ/dlambda per instance; fills ybar_in and xpbar."""
    img = g.batch * g.n * g.n
    prm = RunParams(float(alpha), float(lam), int(tv_iters), 0, 0)
    lb = np.zeros(g.batch)
    vp, vbytes = _ws(vjp_ws)
    _check(load().pnp_unrolled_step_vjp(C.byref(geom(g)), factor, subset, n_subsets, float(eta), C.byref(prm),
                                        float(amom), _ptr(y, img, "y"),
                                        _ptr(b, g.batch * g.n_views * g.n_det, "b"), _ptr(xbar, img, "xbar"),
                                        _ptr(ybar, img, "ybar"), _ptr(ybar_in, img, "ybar_in"),
                                        _ptr(xpbar, img, "xpbar"), lb.ctypes.data_as(C.POINTER(C.c_double)),
                                        _ws(ws)[0], vp, vbytes, _stream(stream)))
    return lb


# ---------------------------------------------------------------- uneven batches, autotuning
def run_many(problems, *, alpha=1.0, lam=0.02, tv_iters=20, momentum=True, stream=None, graph=False,
             kernel_times=False, persistent=False, subset_seed=0):
    """pnp_run_many.  ``problems``: list of dicts with keys plan, stages, eta, seq,
    b, x and optional xtrue, start_iter, y (checkpoint/resume: x and y of
    iteration start_iter in, x and y of the last iteration out); a problem whose
    seq is None takes the library's order drawn from subset_seed for its
    stages.  Returns the list of PSNR logs (None where no xtrue)."""
    arr = (ProblemC * len(problems))()
    keep = []
    logs = []
    for k, pr in enumerate(problems):
        plan = pr["plan"]
        g = plan.g
        plan.ensure_vr_buffer(pr["stages"])
        st = _stages(pr["stages"])
        total = sum(a.iters for a in st)
        eta_a = None if pr.get("eta") is None else (C.c_double * len(st))(*[float(e) for e in pr["eta"]])
        seq_np, seq_p = _seq_ptr(pr.get("seq"), total)
        img = g.batch * g.n * g.n
        xt = pr.get("xtrue")
        log = np.zeros((total, g.batch)) if xt is not None else None
        keep += [st, eta_a, seq_np, log]
        logs.append(log)
        arr[k] = ProblemC(geom(g), st, len(st), eta_a, seq_p,
                          _ptr(pr["b"], g.batch * g.n_views * g.n_det, "b"), _ptr(pr["x"], img, "x"),
                          _ptr(xt, img, "xtrue", True),
                          log.ctypes.data_as(C.POINTER(C.c_double)) if log is not None else None,
                          _ws(plan.ws)[0], int(pr.get("start_iter", 0)),
                          _ptr(pr.get("y"), img, "y", True))
    prm = RunParams(float(alpha), float(lam), int(tv_iters), int(bool(momentum)),
                    _flags(graph, kernel_times, persistent), int(subset_seed) & (2**64 - 1))
    _check(load().pnp_run_many(arr, len(problems), C.byref(prm), _stream(stream)))
    return logs


def autotune(g, stages, ws, *, alpha=1.0, lam=0.02, tv_iters=20, momentum=True, stream=None):
    st = _stages(stages)
    prm = RunParams(float(alpha), float(lam), int(tv_iters), int(bool(momentum)), 0)
    _check(load().pnp_autotune(C.byref(geom(g)), st, len(st), C.byref(prm), _ws(ws)[0], _stream(stream)))
