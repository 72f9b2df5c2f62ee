"""Host-side pieces of the benchmark: the tile-update count its DRAM traffic figures are scaled by,
the scaling itself, and the validation of --forms (no GPU)."""
import subprocess
import sys
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def brute_updates(mt):
    """Trailing updates of the right-looking tiled Cholesky of Sec. 3.2, counted one by one: for every
    finished column J, one SYRK per diagonal tile (I, I) and one GEMM per tile (I, K), J < K < I."""
    c = 0
    for j in range(mt):
        for i in range(j + 1, mt):
            c += 1                      # SYRK on (I, I)
            c += sum(1 for k in range(j + 1, i))  # GEMM on (I, K)
    return c


@pytest.mark.parametrize("mt", [1, 2, 3, 7, 32, 64])
def test_tile_updates_count(mt):
    sys.path.insert(0, ROOT)
    import bench
    assert bench.tile_updates(mt) == brute_updates(mt)


def test_traffic_scaling_reproduces_the_captures():
    sys.path.insert(0, ROOT)
    import bench
    # the capture sizes give the captured bytes back; other sizes scale with the update count
    assert bench.fp64_cholesky_traffic(8192, 256) == pytest.approx(bench.FP64_CHOL_TRAFFIC_MT32_T256)
    assert bench.fp64_cholesky_traffic(16384, 256) == pytest.approx(
        bench.FP64_CHOL_TRAFFIC_MT32_T256 * brute_updates(64) / brute_updates(32))
    assert bench.fp64_cholesky_traffic(8192, 512) is None


def test_forms_option_rejects_unknown_forms():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--forms", "bf16x6,fp16x2"],
                       capture_output=True, text=True, timeout=120)
    assert r.returncode != 0 and "fp16x2" in r.stderr
