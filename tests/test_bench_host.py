"""Host-side logic of bench.py: the roofline classification of the dominant
kernel class and the source-hash check that keeps ncu traffic figures tied to
the kernel they were measured on (no GPU needed)."""
import json
import os

import pytest

import bench


ALU = {"fp64": (1250.0, "measured by st_probe_fma"), "fp32": (80000.0, "measured by st_probe_fma")}


def _stats(name, ms, gbytes, gflops, launches=1):
    return [{"name": name, "ms": ms, "launches": launches, "bytes": gbytes * 1e9, "flops": gflops * 1e9}]


def test_fp64_only_class_uses_fp64_peak_on_the_mixed_path():
    # the refinement residual computes in FP64 on both paths: 0.86 TFLOP/s is 69 % of 1.25, not of the FP32 rate
    st = _stats("st_residual_fp64@1050625", 7.49, 10.77, 6.46)
    r = bench.roofline(st, 6780.0, "measured", "fp32ir", ALU)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["peak"] == pytest.approx(1.25) and "FP64" in r["peak_source"]
    assert r["frac"] == pytest.approx(6.46 / 7.49 / 1.25, rel=1e-9)


def test_fp32_memory_kernel_is_hbm_bound():
    st = _stats("jacobi_smooth@1046529", 1.0, 3.3, 5.0)
    r = bench.roofline(st, 6780.0, "measured", "fp32ir", ALU)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["frac"] == pytest.approx(3300.0 / 6780.0, rel=1e-9)


def test_fp64_compute_kernel_is_alu_bound():
    st = _stats("jacobi_smooth@1046529", 1.0, 0.7, 1.1)
    r = bench.roofline(st, 6780.0, "measured", "fp64", ALU)
    assert r["bound"] == "alu" and r["frac"] == pytest.approx(1.1 / 1.25, rel=1e-9)


def test_dominant_class_is_the_longest_and_share_is_reported():
    st = _stats("a@1", 1.0, 1.0, 0.1) + _stats("b@1", 3.0, 1.0, 0.1, launches=3)
    r = bench.roofline(st, 6780.0, "measured", "fp64", ALU)
    assert r["kernel"] == "b@1" and r["launches"] == 3
    assert r["ms_per_launch"] == pytest.approx(1.0)
    assert r["share_of_profiled_time"] == pytest.approx(0.75)


def _fake_tree(tmp_path, text):
    src = tmp_path / "paper_2606_09688_gb300" / "csrc"
    src.mkdir(parents=True)
    (src / "k.cu").write_text(text)
    (tmp_path / "profiles").mkdir()
    return src


def test_traffic_follows_the_kernel_sources(tmp_path, monkeypatch):
    src = _fake_tree(tmp_path, "kernel v1")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    entry = {"bytes": 123, "sources": ["k.cu"], "sha256": bench.csrc_hash(["k.cu"])}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"bytes_per_launch": {"fp64:x@9": entry}}))
    assert bench.traffic_for("x@9", "fp64") == 123
    assert bench.traffic_for("x@9", "fp32ir") is None  # another precision: not measured
    (src / "k.cu").write_text("kernel v2")
    assert bench.traffic_for("x@9", "fp64") is None  # the kernel changed after the capture


def test_traffic_entry_without_sources_is_ignored(tmp_path, monkeypatch):
    _fake_tree(tmp_path, "kernel")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    entry = {"bytes": 5, "sources": [], "sha256": bench.csrc_hash([])}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"bytes_per_launch": {"fp64:x@9": entry}}))
    assert bench.traffic_for("x@9", "fp64") is None


def test_committed_traffic_file_parses():
    path = os.path.join(bench.ROOT, "profiles", "traffic.json")
    with open(path) as f:
        d = json.load(f)
    assert isinstance(d.get("bytes_per_launch"), dict) and d.get("how")


def test_alu_peak_comes_from_the_probe_figure():
    st = _stats("st_residual_fp64@1050625", 7.49, 10.77, 6.46)
    alu = {"fp64": (1000.0, "measured by st_probe_fma"), "fp32": (70000.0, "measured by st_probe_fma")}
    r = bench.roofline(st, 6780.0, "measured", "fp64", alu)
    assert r["peak"] == pytest.approx(1.0) and r["frac"] == pytest.approx(6.46 / 7.49, rel=1e-9)
    assert "st_probe_fma" in r["peak_source"]


def test_final_line_roofline_is_compact():
    st = _stats("combine_level@1050625", 7.49, 10.77, 6.46) + _stats("jacobi_smooth@1046529", 1.0, 3.3, 5.0)
    r = bench.compact_roofline(bench.roofline(st, 6780.0, "measured", "fp64", ALU))
    assert set(r) == {"bound", "achieved", "peak", "unit", "frac", "traffic", "kernel"}
    assert len(json.dumps(r)) < 200


def test_combination_is_judged_against_hbm():
    # double-single combination: FP32-pipe arithmetic, so the HBM fraction bounds it
    st = _stats("combine_level@1050625", 2.0, 10.77, 7.5)
    r = bench.roofline(st, 6780.0, "measured", "fp64", ALU)
    assert r["bound"] == "hbm" and r["frac"] == pytest.approx(10770.0 / 2.0 / 6780.0, rel=1e-9)
