"""Host logic of the benchmark that needs no GPU: the schedule cut used by the
time-to-PSNR legs."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2203_07308_gb300 import synth  # noqa: E402


def test_cut_schedule_keeps_stages_and_alignment():
    st = [synth.Stage(2, 20, 8), synth.Stage(4, 0, 1, kind=1), synth.Stage(1, 80, 8, estimator=1)]
    cut = bench.cut_schedule(st, 25)
    assert [(s.factor, s.iters, s.n_subsets, s.kind, s.estimator) for s in cut] == \
        [(2, 20, 8, 0, 0), (4, 0, 1, 1, 0), (1, 5, 8, 0, 1)]
    assert [s.iters for s in bench.cut_schedule(st, 10)] == [10, 0, 0]
    assert [s.iters for s in bench.cut_schedule(st, 0)] == [0, 0, 0]
    assert [s.iters for s in bench.cut_schedule(st, 1000)] == [20, 0, 80]
    assert st[2].iters == 80                      # the input schedule is not modified

