"""The launch-list summary used for the committed profiles: kernel names are
shortened (namespace dropped, template arguments kept), device times in any
unit are summed per kernel and shares add up to 100 %."""
import csv

from paper_2404_09373_gb300 import ncu_summary as N


def _write(path, rows):
    with open(path, "w", newline="") as f:
        w = csv.writer(f)
        w.writerow(["ID", "Kernel Name", "Metric Name", "Metric Unit", "Metric Value"])
        for r in rows:
            w.writerow(r)


def test_kernel_name_short_form():
    assert N.kernel_name("void (anonymous namespace)::k_oz_gemm<8, 48>(OzGemmParams)") == "k_oz_gemm<8, 48>"
    assert N.kernel_name("<unnamed>::k_fft_pass<16>(FftPass)") == "k_fft_pass<16>"
    assert N.kernel_name("k_phi(int, int)") == "k_phi"


def test_summary_sums_units_and_shares(tmp_path, capsys):
    p = tmp_path / "launches.csv"
    _write(p, [
        [0, "void (anonymous namespace)::k_oz_gemm<8, 48>(P)", "gpu__time_duration.sum", "ms", "1.5"],
        [1, "void (anonymous namespace)::k_oz_gemm<8, 48>(P)", "gpu__time_duration.sum", "us", "500"],
        [2, "k_phi(int)", "gpu__time_duration.sum", "ns", "2,000,000"],
        [3, "k_phi(int)", "dram__bytes_read.sum", "byte", "123"],
    ])
    N.main(str(p))
    out = capsys.readouterr().out.splitlines()
    rows = {l.split()[0]: l for l in out[1:]}
    gemm = rows["k_oz_gemm<8,"].split()
    assert gemm[-3] == "2" and float(gemm[-2]) == 2.0 and gemm[-1] == "50.00%"
    phi = rows["k_phi"].split()
    assert phi[1] == "1" and float(phi[2]) == 2.0 and phi[3] == "50.00%"
    total = rows["total"].split()
    assert total[1] == "3" and float(total[2]) == 4.0
