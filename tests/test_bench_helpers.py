"""Host-side helpers of bench.py (no GPU): the stored exact values it reads,
the time-to-accuracy projection, the peak lookup and the parsing of the
machine-readable lines of an ncu summary."""
import importlib.util
import math
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", ROOT / "bench.py")
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_golden_readers(bench):
    assert abs(bench.golden_e_lat("cube_128c_n8_q1") - 3.678393512740982) < 1e-15
    assert abs(bench.golden_e_lat("cube_128c_n8_q1", column=9) - 3.627886388286265) < 1e-15
    assert bench.golden_e_lat("no_such_workload") is None
    g = bench.golden_offlattice("offcube_128c_n8_q1")
    assert g["n_pairs"] == 20 and g["e_far"] > 0 and g["continuum"] > g["e_plain"]


def test_time_to_accuracy_scales_as_variance(bench):
    e = bench.golden_e_lat("bench_128c_n4096_pm")
    est = {"mean": e, "stderr": 2e-3 * abs(e), "tau_int": 0.7, "n": 1000}
    r = bench.time_to_accuracy(est, 10.0, 1)
    assert math.isclose(r["projected_seconds"], 40.0, rel_tol=1e-12)  # (2e-3 / 1e-3)^2 x 10 s
    assert r["delta"] == 0.0 and r["samples"] == 1000
    r2 = bench.time_to_accuracy(est, 10.0, 4)
    assert r2["samples"] == 4000
    assert bench.time_to_accuracy({"mean": 0, "stderr": 0.0, "tau_int": 0, "n": 0}, 1.0, 1) is None


def test_measured_peaks_present_or_fallback(bench):
    peak, kind = bench.measured_peaks()
    assert peak > 1000 and kind in ("measured", "fallback")


def test_profiled_traffic_parsing(bench, tmp_path, monkeypatch):
    name = "pass_kernel<float, over-relaxation>"
    f = tmp_path / "summary.txt"
    f.write_text("# comment: not parsed\n"
                 f"kernel: {name}\n"
                 f"kernel_src_sha256_16: {bench.kernel_src_hash()}\n"
                 "dram_bytes_per_launch_full: 12345\n")
    monkeypatch.setitem(bench.PROFILE_TRAFFIC, name, f)
    assert bench.profiled_traffic(name) == 12345.0
    # stale counters (kernel sources changed since) are not reported
    f.write_text(f"kernel: {name}\nkernel_src_sha256_16: 0000000000000000\n"
                 "dram_bytes_per_launch_full: 12345\n")
    assert bench.profiled_traffic(name) is None
    assert bench.profiled_traffic("no such kernel") is None
