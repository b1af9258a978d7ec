"""Host-side pieces of bench.py that decide what its JSON line reports: the
committed ncu traffic line of the metric kernel was taken on the kernel's current
source (else the line's roofline.traffic would be null), and the peak bandwidth
comes from the measured peaks file when it is present."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_traffic_line_matches_the_current_kernel_source():
    import bench
    t = bench.load_traffic("k_ras_apply_fp32_1m")
    assert t is not None, "profiles/k_ras_apply_fp32_1m.md records another source hash"
    # ncu DRAM bytes per launch against the algorithmic 68.56 MB of the 1M workload
    assert 0.9 * 68.56e6 < t < 1.1 * 68.56e6


def test_peak_comes_from_the_measured_file():
    import bench
    peak, kind = bench.load_peaks()
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        assert kind == "measured"
        assert peak == float(json.load(open(path))["hbm_gbs"])
    else:
        assert (peak, kind) == (6800.0, "fallback")
