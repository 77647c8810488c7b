"""Host logic of the benchmark that needs no GPU: the schedule cut used by the
time-to-PSNR legs, the roofline arithmetic and the clock-record summary."""
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



def test_roofline_arithmetic():
    """FP32 peak = SMs x 128 lanes x 2 (FMA) x clock; a projector launch does 12
    FLOP and 16 B of taps per projected sample, a denoise 24 FLOP per pixel and
    FGP iteration; achieved = work / live phase time."""
    onchip = {"l1_gbs": 40000.0, "l2_gbs": 18000.0}
    out, peak = bench.rooflines(samples_step=1e9, pixel_iters_step=1e8, steps=2,
                                ph_ms={"forward": 100.0, "backward": 50.0, "denoise": 20.0, "prep": 1.0},
                                ph_n={"forward": 10, "backward": 10, "denoise": 5, "prep": 10},
                                n_sm=152, clock_mhz=2070.0, onchip=onchip)
    assert abs(peak - 152 * 128 * 2 * 2070e6 / 1e12) < 1e-9
    fw = out["forward"]
    assert abs(fw["alu"]["achieved"] - 12 * 2e9 / 0.1 / 1e12) < 1e-12
    assert abs(fw["l1"]["achieved"] - 16 * 2e9 / 0.1 / 1e9) < 1e-9
    assert abs(fw["l1"]["frac"] - fw["l1"]["achieved"] / 40000.0) < 1e-15
    assert abs(fw["gsamples_per_s"] - 2e9 / 0.1 / 1e9) < 1e-9 and fw["mean_unit_us"] == 10000.0
    assert abs(out["backward"]["alu"]["achieved"] - 12 * 2e9 / 0.05 / 1e12) < 1e-12
    dn = out["denoise"]
    assert abs(dn["alu"]["achieved"] - 24 * 2e8 / 0.02 / 1e12) < 1e-12
    assert abs(dn["gpixel_iters_per_s"] - 2e8 / 0.02 / 1e9) < 1e-9
    assert "prep" not in out
    empty, _ = bench.rooflines(1e9, 1e8, 2, {"forward": 0.0}, {"forward": 0}, 152, 2070.0, onchip)
    assert empty == {}


def test_clock_summary_flags_throttle_reasons(tmp_path):
    """The nvidia-smi record taken during the timed region: median SM clock, the
    maximum clock, and every throttle reason seen Active at least once."""
    path = tmp_path / "clocks.csv"
    path.write_text("\n".join([
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]) + "\n")
    cs = bench.ClockSampler(0)
    cs.path = str(path)
    got = cs.summary()
    assert got == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "samples": 3, "reasons": ["sw_power_cap"]}
    assert not path.exists()
