"""Host-side logic of bench.py that needs no GPU: the source hash that keeps a recorded
ncu traffic figure valid only for the kernel it was taken on, the traffic lookup, and the
summary of the clock samples taken during the timed region."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_source_hash_ignores_comments_and_whitespace_only():
    a = "int f(int x) {\n  return x + 1;  // add one\n}\n"
    b = "/* header */ int f(int x) { return x + 1; }"
    c = "int f(int x) { return x + 2; }"
    assert bench.source_hash(a) == bench.source_hash(b)
    assert bench.source_hash(a) != bench.source_hash(c)


def test_traffic_is_the_recorded_figure_scaled_or_nothing():
    with open(os.path.join(ROOT, "profiles", "tc_corr_traffic.json")) as fh:
        rec = json.load(fh)
    key = next(k for k in rec if not k.startswith("_"))
    workload, dtype = key.split(":")
    got = bench.traffic_from_profile(workload, dtype, 512)
    if rec[key]["src_hash"] == bench.src_hash():
        assert got == rec[key]["bytes_per_frame"] * 512
    else:                       # the kernel changed since the capture: no traffic claimed
        assert got is None
    assert bench.traffic_from_profile(workload, "no_such_dtype", 512) is None
    assert bench.traffic_from_profile("no_such_workload", dtype, 512) is None


def test_clock_summary_keeps_the_window_and_reads_reasons():
    def line(sm, power, hw="Not Active", pc="Not Active"):
        return f"0, {sm}, 2070, {power}, 0x0, {hw}, Not Active, Not Active, {pc}"
    lines = [(0.5, line(1000, 100, hw="Active")),        # before the window: ignored
             (1.0, line(2000, 400)), (1.1, line(2010, 410, pc="Active")),
             (1.2, line(1990, 420)), (1.3, "garbage"),
             (9.0, line(500, 90, hw="Active"))]          # after the window: ignored
    s = bench.ClockSampler.summarize(lines, 1.0, 1.25)
    assert s["samples"] == 3 and s["sm_mhz"] == 2000.0 and s["sm_max_mhz"] == 2070.0
    assert s["power_w_median"] == 410.0
    assert s["reasons"] == ["sw_power_cap"]
    assert bench.ClockSampler.summarize(lines, 5.0, 6.0) is None


def test_nmse_stats_by_hand():
    # four frames of two entries, SNR labels 0, 10, 0, 10; frame f has reference energy 2
    # and error energy e_f, so its NMSE is e_f / 2, and each SNR pools its frames
    import numpy as np
    ref = np.ones((4, 2), dtype=np.complex64)
    est = ref.copy()
    est[0, 0] += 1.0          # e = 1
    est[1, 1] += 2.0j         # e = 4
    est[2, 0] += 0.5          # e = 0.25
    st = bench.nmse_stats(est, ref, [0, 10, 0, 10], chunk=3)   # a chunk boundary inside
    assert st["frames"] == 4
    assert abs(st["nmse"] - (1 + 4 + 0.25) / 8) < 1e-12
    assert abs(st["nmse_by_snr_db"]["0"] - (1 + 0.25) / 4) < 1e-12
    assert abs(st["nmse_by_snr_db"]["10"] - 4 / 4) < 1e-12
    assert abs(st["nmse_worst_frame"] - 2.0) < 1e-12


def test_serving_knee_rule():
    def row(rate, delivered, p99):
        return {"offered_hz": rate, "delivered_frames_per_s": delivered, "p99_ms": p99}
    sweep = [row(10e3, 9.97e3, 0.06), row(20e3, 19.9e3, 0.065), row(40e3, 39.8e3, 0.24),
             row(80e3, 79.8e3, 0.241), row(160e3, 146e3, 170.0)]
    assert bench.knee_of(sweep) == 40e3          # 80k: p99 just above 4x the 10k one
    sweep[3]["p99_ms"] = 0.24
    assert bench.knee_of(sweep) == 80e3
    sweep[3]["delivered_frames_per_s"] = 0.94 * 80e3   # not delivered
    assert bench.knee_of(sweep) == 40e3
    assert bench.knee_of([]) is None
