"""The bench line's roofline arithmetic (no GPU): algorithmic bytes and flops
per launch, the derived ALU peaks, and when recorded DRAM traffic may be
reported."""
import importlib.util
import math
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_algorithmic_bytes_per_launch(bench):
    n = 256 ** 3
    # x pass: src, V, dst read + dst write; strided: src, dst read + dst write (FP32)
    assert bench.algorithmic_bytes("x_pass", n, 4) == 16 * n
    assert bench.algorithmic_bytes("y_pass", n, 4) == 12 * n
    assert bench.algorithmic_bytes("z_pass", n, 4) == 12 * n
    assert bench.algorithmic_bytes("xy_pass", n, 4) == 16 * n
    assert bench.algorithmic_bytes("x_pass", n, 8) == 32 * n
    # a separable potential: the x pass reads no V field
    assert bench.algorithmic_bytes("x_pass", n, 4, True) == 12 * n == 201326592
    assert bench.algorithmic_bytes("y_pass", n, 4, True) == 12 * n
    assert bench.algorithmic_bytes("xy_pass", n, 4, True) == 16 * n


def test_algorithmic_flops_per_launch(bench):
    n = (64, 64, 64)
    N = 64 ** 3
    assert bench.algorithmic_flops("x_pass", n, N) == (5 * 6 + 5) * N
    assert bench.algorithmic_flops("xy_pass", n, N) == 2 * (5 * 6 + 5) * N == 18350080
    assert bench.algorithmic_flops("z_pass", (256, 128, 32), 256 * 128 * 32) == (5 * 5 + 5) * 256 * 128 * 32


def test_alu_peaks(bench):
    # 152 SMs x 128 FP32 lanes x 2 flops x 2070 MHz
    assert math.isclose(bench.alu_peak_tflops(32, 2070.0), 152 * 128 * 2 * 2.07e9 / 1e12)
    assert math.isclose(bench.alu_peak_tflops(32, None), bench.alu_peak_tflops(32, 2070.0))
    assert math.isclose(bench.alu_peak_tflops(64, 2070.0), 1.25)
    assert math.isclose(bench.alu_peak_tflops(64, 1035.0), 0.625)


def test_recorded_traffic_only_for_the_recorded_sources(bench, monkeypatch):
    rec = bench.MEASURED_TRAFFIC["aniso_ho_3d_256"]
    # reported while the sources hash to the recorded value
    monkeypatch.setitem(bench.MEASURED_TRAFFIC, "source_hash", bench.traffic_source_hash())
    assert bench.measured_traffic("aniso_ho_3d_256", "x_pass", 6) == rec["x_pass"][6]
    assert bench.measured_traffic("aniso_ho_3d_256", "y_pass", 0) == rec["y_pass"][0]
    # recorded bytes stay below the algorithmic ones (no re-reads; write-backs land later)
    for k in ("x_pass", "y_pass", "z_pass"):
        for v in rec[k].values():
            assert v < bench.algorithmic_bytes(k, 256 ** 3, 4, True)
    assert bench.measured_traffic("aniso_ho_3d_256", "x_pass", 5) is None      # not recorded
    assert bench.measured_traffic("ho_3d_64_fp32", "x_pass", 0) is None         # not recorded
    monkeypatch.setitem(bench.MEASURED_TRAFFIC, "source_hash", "0000000000000000")
    assert bench.measured_traffic("aniso_ho_3d_256", "x_pass", 6) is None       # kernels changed
