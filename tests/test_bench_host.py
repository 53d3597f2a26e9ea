"""CPU checks of bench.py's host logic: byte and flop models, the source-digest
guard on profiled DRAM traffic, and the clock / throttle-reason summary."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_byte_and_flop_models():
    # per element: 2 (P+1)^3 coefficients + 7 Q^3 geometric factors, FP32
    assert bench.helm_bytes_per_elem(4, 6, 4) == (2 * 125 + 7 * 216) * 4 == 7048
    assert bench.helm_bytes_per_elem(4, 6, 8, dim=2) == (2 * 25 + 4 * 36) * 8
    # sum-factorised BwdTrans twice (forward and transposed) + 6 Q^4 gradient work + 20 Q^3 pointwise
    n, Q = 5, 6
    bwd = n ** 3 * Q + n ** 2 * Q ** 2 + n * Q ** 3
    assert bench.helm_flops_per_elem(4, 6) == 2 * (2 * bwd + 6 * Q ** 4) + 20 * Q ** 3 == 30792


def test_traffic_is_reported_only_for_the_profiled_kernel_source(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    dig = bench.kernel_digest(bench.HELM_SOURCES)
    (prof / "k.txt").write_text(f"# header\nkernel_digest: {dig}\ndram_bytes_per_launch: 123\n")
    (prof / "old.txt").write_text("kernel_digest: 0000000000000000\ndram_bytes_per_launch: 456\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_digest", lambda names=None: dig)
    assert bench.profiled_traffic("k.txt") == 123.0
    assert bench.profiled_traffic("old.txt") is None
    assert bench.profiled_traffic("missing.txt") is None


def test_clock_summary_flags_throttle_reasons():
    c = bench.ClockSampler(0)
    c.lines = ["0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active",
               "0, 1500, 2070, 1390.1, 0x4, Not Active, Not Active, Not Active, Active",
               "0, 2070, 2070, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active",
               "garbage line"]
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
