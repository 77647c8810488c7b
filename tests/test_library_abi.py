"""CPU-side checks of the C ABI: the library builds and loads without a GPU,
exports every function include/pnp_ms2g.h declares, and rejects invalid
arguments on the host before anything is launched."""
import ctypes as C
import math

import numpy as np
import pytest

import paper_2203_07308_gb300 as pnp
from paper_2203_07308_gb300 import _native, build, synth


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _native.load()


def test_exports_every_declared_symbol(lib):
    names = _native.header_functions()
    assert len(names) >= 15
    raw = C.CDLL(_native.LIB_PATH)
    for n in names:
        assert hasattr(raw, n), n


def test_workspace_size_and_invalid_geometry(lib):
    g = synth.make_geometry(256, 360, 512)
    nbytes = pnp.workspace_size(g)
    assert nbytes > 360 * 512 * 24 * 3
    bad = synth.Geometry(n=256, n_views=360, n_det=512, dso=100.0, ddo=100.0, det_pitch=1.0)
    with pytest.raises(pnp.PnpError) as e:
        pnp.workspace_size(bad)
    assert e.value.code == _native.PNP_EINVAL and "source too close" in str(e.value)
    for field, val in [("n", 2), ("n_views", 0), ("det_pitch", 0.0), ("step", -1.0), ("dso", math.inf)]:
        kw = dict(g.__dict__)
        kw[field] = val
        with pytest.raises(pnp.PnpError):
            pnp.workspace_size(synth.Geometry(**kw))


def test_calls_reject_bad_arguments_before_launch(lib):
    g = _native.geom(synth.make_geometry(64, 90, 96))
    null = C.c_void_p(0)
    # unprepared (NULL) workspace, bad factor, bad subset: rejected on the host
    assert lib.pnp_project(C.byref(g), 1, C.c_void_p(16), None, C.c_void_p(16), 0, 1, null, null) == 1
    assert lib.pnp_project(C.byref(g), 3, C.c_void_p(16), None, C.c_void_p(16), 0, 1, C.c_void_p(256), null) == 1
    assert lib.pnp_project(C.byref(g), 1, C.c_void_p(16), None, C.c_void_p(16), 5, 4, C.c_void_p(256), null) == 1
    # a workspace never passed to pnp_setup is reported as such
    assert lib.pnp_project(C.byref(g), 1, C.c_void_p(16), None, C.c_void_p(16), 0, 1, C.c_void_p(4096), null) == 5
    assert "pnp_setup" in pnp.last_error()
    # factor 8 is unavailable at n = 24 (fewer than 4 coarse pixels per side)
    g24 = _native.geom(synth.make_geometry(24, 10, 32))
    assert lib.pnp_sketch(C.byref(g24), 8, C.c_void_p(16), C.c_void_p(16), null) == 1
    assert lib.pnp_tv_denoise(C.c_void_p(16), C.c_void_p(16), 8, 1, C.c_float(0.1), 5, null, 0, null) == 1
    size = C.c_size_t(0)
    assert lib.pnp_tv_workspace_size(64, 2, C.byref(size)) == 0 and size.value == 8 * 2 * 64 * 64 * 4
    assert lib.pnp_launch_count() == 0


def test_estimator_buffer_sizes(lib):
    """pnp_vr_buffer_size: 0 for vanilla schedules (and for SVRG/SAGA stages with
    one subset), five image planes for SVRG, plus P_k level images per instance
    for SAGA's table; factors that do not divide n are rejected."""
    g = synth.make_geometry(64, 60, 96, batch=2)
    img = 2 * 64 * 64 * 4
    assert pnp.vr_buffer_size(g, [synth.Stage(2, 5, 3), synth.Stage(1, 5, 1)]) == 0
    assert pnp.vr_buffer_size(g, [synth.Stage(2, 5, 1, estimator=2)]) == 0
    assert pnp.vr_buffer_size(g, [synth.Stage(2, 5, 3, estimator=1)]) == 5 * img
    saga = pnp.vr_buffer_size(g, [synth.Stage(2, 5, 3, estimator=2), synth.Stage(1, 5, 2, estimator=2)])
    assert saga == 5 * img + max(3 * 2 * 32 * 32 * 4, 2 * img)
    with pytest.raises(pnp.PnpError):
        pnp.vr_buffer_size(g, [synth.Stage(3, 5, 3, estimator=1)])


def test_binding_constants_match_the_header():
    """Every constant the Python binding restates equals the C header's value
    (error codes, sketch kinds, estimators, run flags, phases, launch-shape
    flags, limits), so the two cannot drift apart."""
    import re
    from paper_2203_07308_gb300 import _native as N
    text = open(N.HEADER).read()

    def define(name):
        m = re.search(r"#define\s+%s\s+(.+)" % name, text)
        assert m, name
        expr = m.group(1).split("/*")[0].strip().replace("u <<", " <<").replace("u)", ")")
        return eval(expr, {})                     # plain integer expressions: 0, (1 << 8), (32 << 20)

    codes = {k: int(v) for k, v in re.findall(r"(PNP_E[A-Z]+|PNP_OK)\s*=\s*(\d+)", text)}
    assert codes == {"PNP_OK": N.PNP_OK, "PNP_EINVAL": N.PNP_EINVAL, "PNP_ECUDA": N.PNP_ECUDA,
                     "PNP_ETIMEOUT": N.PNP_ETIMEOUT, "PNP_EUNSUPPORTED": N.PNP_EUNSUPPORTED,
                     "PNP_ESTATE": N.PNP_ESTATE}
    pairs = {"PNP_SKETCH_POOL": N.SKETCH_POOL, "PNP_SKETCH_BICUBIC": N.SKETCH_BICUBIC,
             "PNP_EST_MINIBATCH": N.EST_MINIBATCH, "PNP_EST_SVRG": N.EST_SVRG, "PNP_EST_SAGA": N.EST_SAGA,
             "PNP_RUN_GRAPH": N.RUN_GRAPH, "PNP_RUN_KERNEL_TIMES": N.RUN_KERNEL_TIMES,
             "PNP_RUN_PERSISTENT": N.RUN_PERSISTENT,
             "PNP_BACK_TILE4": N.BACK_TILE4, "PNP_BACK_SCATTER": N.BACK_SCATTER, "PNP_BACK_TABLE": N.BACK_TABLE,
             "PNP_MAX_LOG_ITERS": N.MAX_LOG_ITERS, "PNP_NOALLOC_SCRATCH_BYTES": N.NOALLOC_SCRATCH_BYTES,
             "PNP_N_PHASES": len(N.PHASES)}
    for name, value in pairs.items():
        assert define(name) == value, name
    for k, ph in enumerate(N.PHASES):
        assert define("PNP_PHASE_" + ph.upper()) == k, ph


def test_schedule_walks_algorithm_1(lib):
    """pnp_schedule (host only): iteration i of the schedule belongs to the stage
    whose iterations cover it, takes its subset from the sequence only when that
    stage has P_k > 1, and has the momentum a_i = (i-1)/(i+3) of Sec. 3 (a_1 = 0,
    one global sequence with no restart at stage switches), or 0 without momentum."""
    stages = [synth.Stage(4, 3, 5), synth.Stage(2, 0, 3), synth.Stage(1, 4, 1), synth.Stage(1, 2, 2)]
    seq = [4, 0, 2, 9, 9, 9, 9, 1, 0]
    stage, subset, amom = pnp.schedule(stages, seq, momentum=True)
    assert stage.tolist() == [0, 0, 0, 2, 2, 2, 2, 3, 3]
    assert subset.tolist() == [4, 0, 2, 0, 0, 0, 0, 1, 0]
    for i in range(1, 10):
        assert amom[i - 1] == np.float32((i - 1) / (i + 3))
    assert amom[0] == 0.0
    _, _, a0 = pnp.schedule(stages, seq, momentum=False)
    assert not a0.any()
    with pytest.raises(pnp.PnpError):          # subset id outside its stage's range
        pnp.schedule([synth.Stage(1, 2, 3)], [0, 3])
    with pytest.raises(pnp.PnpError):          # subsets without a sequence
        pnp.schedule([synth.Stage(1, 2, 3)], None)
    total = C.c_int64(0)
    arr = (_native.StageC * 1)(_native.StageC(1, 5, 1, 0, 0))
    i32 = (C.c_int32 * 4)()
    f32 = (C.c_float * 4)()
    assert lib.pnp_schedule(arr, 1, None, 1, i32, i32, f32, 4, C.byref(total)) == _native.PNP_EINVAL
    assert total.value == 5 and "capacity" in pnp.last_error()


def test_subset_sequence_matches_the_oracle(lib):
    """pnp_subset_sequence (host only) draws the same subset order as the
    oracle's independent SplitMix64 / Fisher-Yates restatement, bit for bit, for
    mixed schedules (P = 1 stages, short last epochs, P up to n_views) and
    seeds including 2^64 - 1; counts and argument errors are reported."""
    import oracle
    cases = [([synth.Stage(4, 30, 12), synth.Stage(2, 7, 1), synth.Stage(1, 41, 8)], 7308),
             ([synth.Stage(1, 100, 2)], 0),
             ([synth.Stage(2, 13, 5), synth.Stage(1, 0, 9), synth.Stage(1, 400, 360)], 2**64 - 1),
             ([synth.Stage(1, 5, 1)], 12345)]
    for stages, seed in cases:
        got = pnp.subset_sequence(stages, seed)
        ref = oracle.subset_sequence(stages, seed)
        assert got.dtype == np.int32 and np.array_equal(got, ref), (stages, seed)
    total = C.c_int64(0)
    arr = (_native.StageC * 2)(_native.StageC(1, 5, 3, 0, 0), _native.StageC(1, 4, 2, 0, 0))
    assert lib.pnp_subset_sequence(arr, 2, 1, None, 0, C.byref(total)) == _native.PNP_EINVAL
    assert total.value == 9 and "capacity" in pnp.last_error()
    bad = (_native.StageC * 1)(_native.StageC(1, 5, 0, 0, 0))
    assert lib.pnp_subset_sequence(bad, 1, 1, None, 0, C.byref(total)) == _native.PNP_EINVAL
    with pytest.raises(pnp.PnpError):
        pnp.subset_sequence([synth.Stage(1, -1, 2)], 3)


def test_step_sizes_and_bandwidth_reject_bad_arguments(lib):
    g = _native.geom(synth.make_geometry(64, 90, 96))
    st = (_native.StageC * 1)(_native.StageC(3, 5, 1, 0, 0))
    eta = (C.c_double * 1)()
    null = C.c_void_p(0)
    assert lib.pnp_step_sizes(C.byref(g), st, 1, eta, C.c_void_p(256), null) == _native.PNP_EINVAL   # factor 3
    st[0] = _native.StageC(2, 5, 1, 0, 0)
    assert lib.pnp_step_sizes(C.byref(g), st, 1, eta, C.c_void_p(4096), null) == _native.PNP_ESTATE
    out = (C.c_double * 3)()
    assert lib.pnp_onchip_bandwidth(C.c_void_p(256), 1 << 20, out, null) == _native.PNP_EINVAL
    assert "needs" in pnp.last_error()
