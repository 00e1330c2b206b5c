"""Summarise an ncu launch list (--metrics gpu__time_duration.sum --csv) per kernel.

    python profiles/summarize_launches.py launches.csv
"""
import collections
import csv
import sys

SCALE = {"ns": 1e-3, "nsecond": 1e-3, "us": 1.0, "usecond": 1.0, "ms": 1e3, "msecond": 1e3}


def main(path):
    rows = list(csv.reader(open(path)))
    hdr = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
    h = rows[hdr]
    ki, mi, vi, ui = (h.index(k) for k in ("Kernel Name", "Metric Name", "Metric Value", "Metric Unit"))
    agg = collections.defaultdict(lambda: [0, 0.0])
    for r in rows[hdr + 1:]:
        if len(r) > vi and r[mi] == "gpu__time_duration.sum":
            name = r[ki].split("(")[0].replace("<unnamed>::", "")
            agg[name][0] += 1
            agg[name][1] += float(r[vi].replace(",", "")) * SCALE[r[ui]]
    tot = sum(v[1] for v in agg.values())
    print(f"launches {sum(v[0] for v in agg.values())}, total {tot / 1e3:.1f} ms (serialised, cold cache)")
    print(f"| kernel | launches | total ms | share | avg us |\n|---|---|---|---|---|")
    for k, (c, t) in sorted(agg.items(), key=lambda x: -x[1][1]):
        if t / tot >= 0.001:
            print(f"| {k} | {c} | {t / 1e3:.2f} | {100 * t / tot:.1f}% | {t / c:.1f} |")


if __name__ == "__main__":
    main(sys.argv[1])
