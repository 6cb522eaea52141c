"""Host arithmetic of the benchmark line (no GPU): the flop counts per pair,
the roofline fractions, and the rule that DRAM traffic is read from a
committed ncu summary only while the kernel's source is unchanged."""
import hashlib
import os

import pytest

import bench


def test_flops_per_pair_of_the_nine_column_applies():
    # kernel evaluation plus 2 flops per accumulator: A has 2 + 4 k accumulators
    # per target (area and W_V for the high-order part, area and W_U for B0)
    assert bench.flops_per_pair("apply_A", {"launches": 2, "columns": 18}) == 26 + 2 * (2 + 36)
    assert bench.flops_per_pair("apply_L", {"launches": 1, "columns": 9}) == 9 + 2 * (1 + 9)
    # no column count recorded: the 3-column kernel
    assert bench.flops_per_pair("apply_A", {"launches": 1}) == 26 + 2 * (2 + 12)
    assert bench.flops_per_pair("energy_direct", {}) == 20
    assert bench.flops_per_pair("chol_solve", {}) is None


def _fake_root(tmp_path, src_text, recorded_hash, traffic=123456):
    csrc = tmp_path / "paper_2107_01664_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "pairs.cu").write_text(src_text)
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "apply_A_torus_20k.txt").write_text(
        "# ncu summary\nkernel: k_apply_wide\nsource_sha256: %s\ndram_bytes_per_launch: %d\n" % (recorded_hash, traffic))
    return str(tmp_path)


def test_profile_traffic_only_while_the_source_matches(tmp_path, monkeypatch):
    src = "// kernel source\n"
    good = hashlib.sha256(src.encode()).hexdigest()
    root = _fake_root(tmp_path, src, good)
    monkeypatch.setattr(bench, "ROOT", root)
    assert bench.profile_traffic("apply_A", "torus_20k") == 123456.0
    # the kernel's file changed after the capture: no traffic figure
    (tmp_path / "paper_2107_01664_gb300" / "csrc" / "pairs.cu").write_text(src + "// edited\n")
    assert bench.profile_traffic("apply_A", "torus_20k") is None
    # no summary for that workload
    assert bench.profile_traffic("apply_A", "icosphere_l8") is None


def test_hbm_roofline_arithmetic(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))          # no summaries: traffic None
    monkeypatch.setattr(bench, "measured_peaks", lambda: ({"hbm_gbs": 5000.0}, "measured"))
    stat = {"launches": 4, "ms": 8.0, "units": 4 * 1000.0}   # 2 ms and 1000 units per launch
    r = bench.kernel_roofline("cg", stat, None, "torus_20k", None, bytes_per_unit=2.0e6)
    assert r["ms_per_launch"] == pytest.approx(2.0)
    assert r["achieved"] == pytest.approx(2.0e6 * 1000 / 2e-3 / 1e9)   # 1000 GB/s
    assert r["frac"] == pytest.approx(0.2)
    assert r["bound"] == "hbm" and r["traffic"] is None


def test_alu_roofline_against_the_fp32_peak(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "fp32_peak_tflops", lambda dev: (80.0, "test peak"))
    stat = {"launches": 1, "ms": 1.0, "units": 4.0e8}
    r = bench.kernel_roofline("apply_A", stat, 100, "torus_20k", None)
    assert r["achieved"] == pytest.approx(100 * 4.0e8 / 1e-3 / 1e12)   # 40 TFLOP/s
    assert r["frac"] == pytest.approx(0.5)
    assert r["unit"] == "TFLOP/s"


def test_committed_summaries_name_their_command_and_source():
    prof = os.path.join(os.path.dirname(bench.__file__), "profiles")
    names = [n for n in os.listdir(prof) if n.endswith(".txt")]
    assert names
    for n in names:
        text = open(os.path.join(prof, n)).read()
        assert "# command: ncu " in text and "--clock-control none" in text, n
        if not n.startswith("launches_"):
            assert "source_sha256:" in text, n
