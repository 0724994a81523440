"""Summarise an ncu --csv launch list (gpu__time_duration.sum) per kernel.

Usage: python -m paper_1412_3784_gb300.summarize_launches launches.csv
Prints launches, total time and share per kernel (markdown table).
"""
import collections
import csv
import sys

UNIT = {"ns": 1e-3, "nsecond": 1e-3, "us": 1.0, "usecond": 1.0, "ms": 1e3, "msecond": 1e3}


def main(path):
    hdr, agg = None, collections.defaultdict(lambda: [0, 0.0])
    for r in csv.reader(open(path)):
        if r and r[0] == "ID":
            hdr = r
            continue
        if not hdr or len(r) != len(hdr):
            continue
        d = dict(zip(hdr, r))
        if d["Metric Name"] != "gpu__time_duration.sum":
            continue
        name = d["Kernel Name"].split("(")[0].replace("void ", "")
        us = float(d["Metric Value"].replace(",", "")) * UNIT[d["Metric Unit"]]
        agg[name][0] += 1
        agg[name][1] += us
    tot = sum(v[1] for v in agg.values())
    print("| kernel | launches | total (us) | per launch (us) | share |")
    print("|---|---|---|---|---|")
    for k, (n, us) in sorted(agg.items(), key=lambda x: -x[1][1]):
        print(f"| `{k}` | {n} | {us:.1f} | {us / n:.1f} | {100 * us / tot:.2f}% |")


if __name__ == "__main__":
    main(sys.argv[1])
