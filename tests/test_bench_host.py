"""Host-side bookkeeping of bench.py (no GPU): the DRAM-traffic lookup that fills
roofline.traffic and the per-kernel table of the LOBPCG line."""
import json

import bench


def _write_capture(path, digest, kernels):
    body = json.dumps({"source_digest": digest, "kernels": kernels})
    path.write_text("# capture\n\n```json\n" + body + "\n```\n")


def test_traffic_scales_the_captured_ratio_by_this_runs_bytes_per_launch(tmp_path, monkeypatch):
    f = tmp_path / "dram_traffic.md"
    _write_capture(f, bench.source_digest(),
                   {"k": {"dram_bytes_per_algorithmic_byte": 0.5}})
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    t, src = bench.measured_traffic("k", {"bytes": 4.0e9, "launches": 8, "ms": 1.0})
    assert t == 0.5 * 4.0e9 / 8
    assert src.endswith("dram_traffic.md")


def test_traffic_is_null_for_other_sources_or_kernels(tmp_path, monkeypatch):
    f = tmp_path / "dram_traffic.md"
    _write_capture(f, "0000000000000000", {"k": {"dram_bytes_per_algorithmic_byte": 0.5}})
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    assert bench.measured_traffic("k", {"bytes": 1.0, "launches": 1})[0] is None
    _write_capture(f, bench.source_digest(), {"k": {"dram_bytes_per_algorithmic_byte": 0.5}})
    assert bench.measured_traffic("other", {"bytes": 1.0, "launches": 1})[0] is None
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "absent.md"))
    assert bench.measured_traffic("k", {"bytes": 1.0, "launches": 1})[0] is None


def test_committed_capture_is_well_formed():
    text = open(bench.TRAFFIC_FILE).read()
    d = json.loads(text.split("```json", 1)[1].split("```", 1)[0])
    assert len(d["source_digest"]) == 16
    for k, v in d["kernels"].items():
        assert v["dram_bytes"] > 0 and v["algorithmic_bytes"] > 0
        assert abs(v["dram_bytes_per_algorithmic_byte"] -
                   v["dram_bytes"] / v["algorithmic_bytes"]) < 1e-3


def test_kernel_table_orders_by_time_and_skips_phases():
    prof = {"a": {"ms": 10.0, "launches": 4}, "phase:gram": {"ms": 99.0, "launches": 1},
            "b": {"ms": 30.0, "launches": 2}}
    t = bench.kernel_table(prof, steps=2)
    assert list(t) == ["b", "a"]
    assert t["b"] == {"ms": 15.0, "launches": 1.0, "share": 0.75}
    assert t["a"]["share"] == 0.25
