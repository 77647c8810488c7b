"""GB300-native (sm_103a) hot path of PnP-MS2G (arXiv 2203.07308).

The numerical path lives in ``libpnp_ms2g.so`` (CUDA kernels behind the C ABI
of ``include/pnp_ms2g.h``); ``_native`` is its ctypes binding, ``synth`` the
seeded input generators.  Build the library with
``python -m paper_2203_07308_gb300.build``.
"""
from . import synth  # noqa: F401
from ._native import (  # noqa: F401
    Geom, Plan, PnpError, backproject, full_grad, full_grad_noalloc,
    header_functions, kernel_times, launch_count, last_error, load,
    objective, onchip_bandwidth, power_iter, project, run, run_many, autotune, sample_count, schedule, setup,
    sketch, sketch_grad, step_sizes, subset_sequence, subset_views,
    tv_denoise, tv_workspace_size, upsample, vr_buffer_size, workspace_size,
)
