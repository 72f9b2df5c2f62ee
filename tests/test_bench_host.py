"""Host-side pieces of the benchmark (no GPU): DRAM traffic is reported only for the launches it was
captured on, never scaled (it grows faster than the tile updates), and --forms rejects unknown forms."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_traffic_only_where_captured():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.fp64_cholesky_traffic(32768, 256) == pytest.approx(bench.FP64_CHOL_TRAFFIC_N32768_T256)
    for n, t in ((16384, 256), (8192, 256), (32768, 512)):
        assert bench.fp64_cholesky_traffic(n, t) is None
    r = bench.mixed_cholesky_roofline(32768, 128, 0.13, "fp32")
    assert r["traffic"] == pytest.approx(bench.MIXED_CHOL_TRAFFIC_N32768_T128)
    assert bench.mixed_cholesky_roofline(16384, 128, 0.05, "fp32")["traffic"] is None
    assert bench.mixed_cholesky_roofline(32768, 128, 0.17, "bf16x6")["traffic"] is None


def test_forms_option_rejects_unknown_forms():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--forms", "bf16x6,fp16x2"],
                       capture_output=True, text=True, timeout=120)
    assert r.returncode != 0 and "fp16x2" in r.stderr
