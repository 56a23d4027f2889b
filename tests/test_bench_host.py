"""Host-side logic of the benchmark that needs no GPU: the serving sweep's sustained rate and
the derived FP32 peak."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _window(rate, done, requests, waiting):
    return {"rate": rate, "assign_done": done, "assign_requests": requests, "fit_deferred_fraction": waiting}


def test_sustained_rate_is_the_largest_rate_within_both_limits():
    sweep = [_window(50, 449, 449, 0.06), _window(100, 954, 954, 0.155), _window(250, 2296, 2296, 0.6)]
    assert bench.sustained_rate(sweep) == 50
    assert bench.sustained_rate(sweep, max_waiting=0.2) == 100
    # an unserved assignment disqualifies a rate even with no job waiting
    sweep.append(_window(500, 4521, 4522, 0.0))
    assert bench.sustained_rate(sweep, max_waiting=0.2) == 100
    # a window without clustering jobs (no fraction) counts as none waiting
    assert bench.sustained_rate([_window(10, 5, 5, None)]) == 10
    assert bench.sustained_rate([_window(10, 4, 5, 0.0)]) is None
    assert bench.sustained_rate([]) is None


def test_derived_fp32_peak_follows_the_sm_count():
    p152 = bench.peaks(152)
    p76 = bench.peaks(76)
    assert abs(p152["fp32_tflops"] - 2 * p76["fp32_tflops"]) < 1e-9
    # 152 SMs x 128 lanes x 2 flop x the maximum SM clock
    mhz = p152["sm_max_mhz"] if "sm_max_mhz" in p152 else 2070.0
    assert abs(p152["fp32_tflops"] - 152 * 128 * 2 * mhz * 1e6 / 1e12) < 1e-6
    assert "152 SMs" in p152["fp32_source"]
