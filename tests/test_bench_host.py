"""Host-side bookkeeping of bench.py (no GPU): the headline's convergence rule, the DRAM-traffic
lookup that fills roofline.traffic, the roofline classification and the per-kernel table."""
import json
import os

import numpy as np
import pytest

import bench


def test_converged_from_needs_every_wanted_state_to_stay_within_tolerance():
    ref = np.array([1.0, 2.0, 3.0])
    hist = np.array([[1.5, 2.5, 3.5, 9.0],      # iteration 0: none within 0.1
                     [1.0, 2.05, 3.5, 9.0],     # 1: two
                     [1.0, 2.0, 3.09, 9.0],     # 2: all three (the guard vector is ignored)
                     [1.0, 2.2, 3.0, 9.0],      # 3: leaves again
                     [1.0, 2.0, 3.0, 7.0],      # 4: all
                     [1.01, 2.0, 3.0, 5.0]])    # 5: all
    first, counts = bench.converged_from(hist, ref, 3)
    assert first == 4
    assert list(counts) == [0, 2, 3, 2, 3, 3]
    iter_ms = np.array([10.0, 20.0, 30.0, 40.0, 50.0, 60.0])
    v, k, n, sec, ok = bench.eigenstates_per_second(hist, ref, iter_ms, 3)
    assert (k, n, ok) == (4, 3, True) and sec == 0.05 and v == pytest.approx(60.0)


def test_unconverged_run_counts_the_states_within_tolerance_at_the_last_step():
    ref = np.array([1.0, 2.0])
    hist = np.array([[1.5, 2.5], [1.0, 2.5]])
    v, k, n, sec, ok = bench.eigenstates_per_second(hist, ref, np.array([5.0, 10.0]), 2)
    assert (k, n, ok) == (1, 1, False) and v == pytest.approx(100.0)


def test_reference_convergence_rule():
    assert bench.reference_converged([[1.0, 2.0], [1.0, 2.005]], 2)
    assert not bench.reference_converged([[1.0, 2.0], [1.0, 2.02]], 2)
    assert bench.reference_converged([[1.0, 2.0, 5.0], [1.0, 2.0, 9.0]], 2)   # guard ignored
    assert not bench.reference_converged([[1.0, 2.0]], 2)


def _write_capture(path, digest, kernels):
    path.write_text(json.dumps({"source_digest": digest, "kernels": kernels}))


def test_traffic_scales_the_captured_ratio_by_this_runs_flops_per_launch(tmp_path):
    f = tmp_path / "dram_traffic.json"
    _write_capture(f, bench.source_digest(), {"k": {"dram_bytes_per_flop": 0.25}})
    t, src = bench.measured_traffic("k", {"flops": 8.0e9, "launches": 8, "ms": 1.0}, str(f))
    assert t == 0.25 * 8.0e9 / 8
    assert src.endswith("dram_traffic.json")


def test_traffic_is_null_for_other_sources_or_kernels(tmp_path):
    f = tmp_path / "dram_traffic.json"
    _write_capture(f, "0000000000000000", {"k": {"dram_bytes_per_flop": 0.5}})
    assert bench.measured_traffic("k", {"flops": 1.0, "launches": 1}, str(f))[0] is None
    _write_capture(f, bench.source_digest(), {"k": {"dram_bytes_per_flop": 0.5}})
    assert bench.measured_traffic("other", {"flops": 1.0, "launches": 1}, str(f))[0] is None
    assert bench.measured_traffic("k", {"flops": 1.0, "launches": 1},
                                  str(tmp_path / "absent.json"))[0] is None


def test_committed_capture_is_well_formed():
    if not os.path.exists(bench.TRAFFIC_FILE):
        pytest.skip("no DRAM capture committed")
    d = json.load(open(bench.TRAFFIC_FILE))
    assert len(d["source_digest"]) == 16
    for k, v in d["kernels"].items():
        assert v["dram_bytes"] > 0 and v["flops"] > 0
        assert abs(v["dram_bytes_per_flop"] - v["dram_bytes"] / v["flops"]) < 1e-6 * max(
            1.0, v["dram_bytes_per_flop"])


def test_roofline_classifies_by_intensity_and_reports_the_tensor_fraction():
    mp = bench.machine_peaks(152, {"sm_max_mhz": 2070.0, "bf16_tflops": 1900.0,
                                   "hbm_gbs": 6800.0})
    assert mp["fp32_tflops"] == pytest.approx(152 * 128 * 2 * 2.07e9 / 1e12)
    # compute-heavy float32 kernel: 40 TFLOP/s, far above the machine balance
    prof = {"level": {"ms": 1000.0, "launches": 10, "flops": 40e12, "bytes": 1e9},
            "small": {"ms": 1.0, "launches": 1, "flops": 1.0, "bytes": 1.0},
            "phase:gram": {"ms": 5000.0, "launches": 1, "flops": 0.0, "bytes": 0.0}}
    rl = bench.roofline_of(prof, mp)
    assert rl["kernel"] == "level" and rl["bound"] == "alu" and rl["unit"] == "TFLOP/s"
    assert rl["frac"] == pytest.approx(40.0 / mp["fp32_tflops"])
    assert rl["frac_of_tensor_peak"] == pytest.approx(40.0 / mp["tf32x3_tflops"])
    # streaming kernel: bound by HBM
    prof = {"copy": {"ms": 1000.0, "launches": 2, "flops": 1e9, "bytes": 3.4e12}}
    rl = bench.roofline_of(prof, mp)
    assert rl["bound"] == "hbm" and rl["achieved"] == pytest.approx(3400.0)
    assert rl["frac"] == pytest.approx(0.5)


def test_kernel_table_orders_by_time_and_skips_phases():
    prof = {"a": {"ms": 10.0, "launches": 4}, "phase:gram": {"ms": 99.0, "launches": 1},
            "b": {"ms": 30.0, "launches": 2}}
    t = bench.kernel_table(prof, steps=2)
    assert list(t) == ["b", "a"]
    assert t["b"] == {"ms": 15.0, "launches": 1.0, "share": 0.75}
    assert t["a"]["share"] == 0.25


def test_source_digest_ignores_comments_and_blank_space_but_not_code():
    a = "int f(int x) {  // doubled\n  return 2 * x; /* twice */ }\n"
    b = "int f(int x) { return 2 * x; }"
    c = "int f(int x) { return 3 * x; }"
    assert bench.source_digest([a]) == bench.source_digest([b])
    assert bench.source_digest([b]) != bench.source_digest([c])
    assert bench._code_only('p = "a//b"; // c') == 'p = "a//b";'
