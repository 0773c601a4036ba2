"""Summarise an ncu launch list (gpu__time_duration.sum per launch, --csv) by kernel.

Usage: python -m paper_2404_09373_gb300.ncu_summary launches.csv
Prints per kernel: launches, total device time, share of the total.
"""
import collections
import csv
import re
import sys


def kernel_name(raw):
    """Short name with template arguments: k_oz_gemm<8, 48>, regular_fft."""
    for ns in ("(anonymous namespace)::", "<unnamed>::", "unnamed>::"):
        raw = raw.replace(ns, "")
    m = re.match(r"\s*(?:void\s+)?([\w:]+(?:<[^()]*>)?)", raw)
    return m.group(1).split("::")[-1] if m else raw


UNIT_NS = {"nsecond": 1.0, "ns": 1.0, "usecond": 1e3, "us": 1e3, "msecond": 1e6, "ms": 1e6, "second": 1e9, "s": 1e9}


def main(path):
    rows = list(csv.reader(open(path)))
    hi = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
    h = rows[hi]
    ik, iv, imn = h.index("Kernel Name"), h.index("Metric Value"), h.index("Metric Name")
    iu = h.index("Metric Unit") if "Metric Unit" in h else None
    agg = collections.defaultdict(lambda: [0, 0.0])
    for r in rows[hi + 1:]:
        if len(r) <= iv or r[imn] != "gpu__time_duration.sum":
            continue
        a = agg[kernel_name(r[ik])]
        a[0] += 1
        scale = UNIT_NS.get(r[iu].strip(), 1.0) if iu is not None else 1.0
        a[1] += float(r[iv].replace(",", "")) * scale  # nanoseconds
    tot = sum(v[1] for v in agg.values())
    print(f"{'kernel':34s} {'launches':>9s} {'total ms':>12s} {'share':>7s}")
    for k, v in sorted(agg.items(), key=lambda kv: -kv[1][1]):
        print(f"{k:34s} {v[0]:9d} {v[1] / 1e6:12.2f} {100 * v[1] / tot:6.2f}%")
    print(f"{'total':34s} {sum(v[0] for v in agg.values()):9d} {tot / 1e6:12.2f}")


if __name__ == "__main__":
    main(sys.argv[1])
