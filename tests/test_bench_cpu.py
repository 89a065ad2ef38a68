"""Host logic of bench.py (no GPU): where the roofline's peak and DRAM traffic come from.

* `traffic` is taken from the committed ncu summary only when that summary was captured on the
  kernel the run used and on the current kernel sources (digest of the sweep sources);
* the peak is the measured HBM copy bandwidth when its file exists, else the stated fallback.
"""

import json
import os

import pytest


@pytest.fixture()
def bench_mod():
    import bench
    return bench


def _write_sources(root, bench, text):
    csrc = os.path.join(root, "paper_1701_04900_gb300", "csrc")
    os.makedirs(csrc, exist_ok=True)
    for f in bench.SWEEP_SOURCES:
        with open(os.path.join(csrc, f), "w") as fh:
            fh.write(f"// {f}\n{text}\n")


def test_sweep_digest_follows_every_sweep_source(tmp_path, monkeypatch, bench_mod):
    monkeypatch.setattr(bench_mod, "ROOT", str(tmp_path))
    _write_sources(str(tmp_path), bench_mod, "v1")
    d1 = bench_mod.sweep_kernel_digest()
    assert d1 == bench_mod.sweep_kernel_digest() and len(d1) == 16
    for f in bench_mod.SWEEP_SOURCES:
        p = os.path.join(str(tmp_path), "paper_1701_04900_gb300", "csrc", f)
        with open(p, "a") as fh:
            fh.write("// changed\n")
        assert bench_mod.sweep_kernel_digest() != d1, f
        _write_sources(str(tmp_path), bench_mod, "v1")
        assert bench_mod.sweep_kernel_digest() == d1


def test_traffic_only_for_its_kernel_and_sources(tmp_path, monkeypatch, bench_mod):
    monkeypatch.setattr(bench_mod, "ROOT", str(tmp_path))
    kernel = "sweep_async_rc_kernel<float, 5> (register increment, column held in registers)"
    assert bench_mod.profile_traffic(kernel) is None  # no summary at all
    os.makedirs(os.path.join(str(tmp_path), "profiles"))
    with open(os.path.join(str(tmp_path), "profiles", "sweep_async_traffic.json"), "w") as fh:
        json.dump({"kernel": "sweep_async_rc_kernel<float, 5>", "kernel_digest": "0123456789abcdef",
                   "dram_bytes_per_sweep": 8.0e9}, fh)
    monkeypatch.setattr(bench_mod, "sweep_kernel_digest", lambda: "0123456789abcdef")
    assert bench_mod.profile_traffic(kernel)["dram_bytes_per_sweep"] == 8.0e9
    assert bench_mod.profile_traffic("sweep_kernel<float, async> (staged residual tile)") is None
    monkeypatch.setattr(bench_mod, "sweep_kernel_digest", lambda: "fedcba9876543210")
    assert bench_mod.profile_traffic(kernel) is None


def test_peak_is_measured_when_recorded(tmp_path, monkeypatch, bench_mod):
    monkeypatch.setattr(bench_mod, "ROOT", str(tmp_path))
    assert bench_mod.measured_peaks() == (6800.0, "fallback")
    with open(os.path.join(str(tmp_path), "MEASURED_PEAKS.json"), "w") as fh:
        json.dump({"hbm_gbs": 6790.7, "bf16_tflops": 1930.6}, fh)
    assert bench_mod.measured_peaks() == (6790.7, "measured")
