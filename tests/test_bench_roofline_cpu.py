"""bench.py's roofline arithmetic on CPU: the dominant kernel family is picked by
time, achieved = algorithmic work per launch / average launch time, frac =
achieved / peak, and the DRAM traffic per launch follows the measured ratio of
that family (null where no capture of the current kernel exists)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _fake_peaks(monkeypatch):
    monkeypatch.setattr(bench, "peaks", lambda: {"hbm_gbs": 5000.0, "bf16_tflops": 2000.0})


def test_hbm_family_dominant(monkeypatch):
    _fake_peaks(monkeypatch)
    monkeypatch.setattr(bench, "TRAFFIC_PER_WORK", {"select_gemm": 2.0})
    kern = {
        "select_gemm": {"launches": 10, "ms": 40.0, "work": 1.0e11, "unit": "byte"},
        "coulomb_V": {"launches": 0, "ms": 20.0, "work": 1.0e15, "unit": "flop"},
    }
    _, roof = bench.roofline(kern, 1)
    assert roof["kernel"] == "select_gemm" and roof["bound"] == "hbm"
    per_launch = 1.0e10
    achieved = per_launch / 4.0e-3 / 1e9  # GB/s
    assert roof["achieved"] == pytest.approx(achieved)
    assert roof["frac"] == pytest.approx(achieved / 5000.0)
    assert roof["traffic"] == pytest.approx(bench.TRAFFIC_PER_WORK["select_gemm"] * per_launch)
    assert roof["avg_launch_ms"] == pytest.approx(4.0)


def test_tensor_family_dominant(monkeypatch):
    _fake_peaks(monkeypatch)
    kern = {"coulomb_V": {"launches": 0, "ms": 50.0, "work": 1.0e14, "unit": "flop"}}
    _, roof = bench.roofline(kern, 1)
    assert roof["bound"] == "tensor" and roof["unit"] == "TFLOP/s"
    achieved = 1.0e14 / 50.0e-3 / 1e12  # one launch counted when none were recorded
    assert roof["achieved"] == pytest.approx(achieved)
    assert roof["tensor_issue_frac"] == pytest.approx(achieved * bench.TC_KERNELS["coulomb_V"] / 2000.0)
    assert roof["traffic"] is None


def test_fp64_simt_family_on_the_plain_path(monkeypatch):
    _fake_peaks(monkeypatch)
    kern = {"fit_zc": {"launches": 2, "ms": 100.0, "work": 2.0e11, "unit": "flop"}}
    _, roof = bench.roofline(kern, 0)
    assert roof["bound"] == "alu" and roof["peak"] == 1.25
    assert roof["achieved"] == pytest.approx(1.0e11 / 50.0e-3 / 1e12)


def _write_launches(path, rows):
    import csv

    with open(path, "w", newline="") as f:
        w = csv.writer(f)
        w.writerow(["ID", "Kernel Name", "Metric Name", "Metric Unit", "Metric Value"])
        for r in rows:
            w.writerow(r)


def test_kernel_name_short_form():
    assert bench.kernel_name("void (anonymous namespace)::k_oz_gemm<8, 48>(OzGemmParams)") == "k_oz_gemm<8, 48>"
    assert bench.kernel_name("<unnamed>::k_fft_pass<16>(FftPass)") == "k_fft_pass<16>"
    assert bench.kernel_name("k_phi(int, int)") == "k_phi"


def test_launch_summary_sums_units_and_shares(tmp_path):
    p = tmp_path / "launches.csv"
    _write_launches(p, [
        [0, "void (anonymous namespace)::k_oz_gemm<8, 48>(P)", "gpu__time_duration.sum", "ms", "1.5"],
        [1, "void (anonymous namespace)::k_oz_gemm<8, 48>(P)", "gpu__time_duration.sum", "us", "500"],
        [2, "k_phi(int)", "gpu__time_duration.sum", "ns", "2,000,000"],
        [3, "k_phi(int)", "dram__bytes_read.sum", "byte", "123"],
    ])
    rows = {r[0]: r for r in bench.launch_summary(str(p))}
    assert rows["k_oz_gemm<8, 48>"][1:] == (2, pytest.approx(2.0), pytest.approx(0.5))
    assert rows["k_phi"][1:] == (1, pytest.approx(2.0), pytest.approx(0.5))
