"""Host arithmetic of the benchmark's roofline objects (CPU only)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_alu_roofline_arithmetic():
    r = bench.alu_roofline(10.0, 5_033_654, 1.94e-3, 152, 2070.0)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["flops_per_unit"] == 181 * 10 + 12
    assert abs(r["peak"] - 152 * 128 * 2 * 2.07e9 / 1e12) < 0.01          # 80.55 TFLOP/s
    assert abs(r["achieved"] - 1822 * 5_033_654 / 1.94e-3 / 1e12) < 1e-3
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-3


def test_committed_profiles_parse():
    """Every committed ncu summary that carries a source hash carries its
    per-unit figure as a number (what the benchmark reads)."""
    import glob
    import re
    for path in glob.glob(os.path.join(ROOT, "profiles", "*.md")):
        txt = open(path).read()
        if "kernel_source_sha256_16:" in txt:
            assert re.search(r"kernel_source_sha256_16:\s*[0-9a-f]{16}\b", txt), path
            assert re.search(r"dram_bytes_per_unit:\s*[0-9.]+", txt), path
