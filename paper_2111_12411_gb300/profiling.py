"""Summarise an ncu launch list (``--metrics gpu__time_duration.sum --csv``):
launches, total time and share per kernel.  Usage: python -m paper_2111_12411_gb300.profiling launches.csv"""
import collections
import csv
import sys

SCALE = {"ns": 1e-6, "nsecond": 1e-6, "us": 1e-3, "usecond": 1e-3, "ms": 1.0, "msecond": 1.0, "s": 1e3, "second": 1e3}


def summarize(path):
    rows = [r for r in csv.reader(open(path)) if len(r) > 10]
    hdr = rows[0]
    ki, mi, vi, ui = (hdr.index(k) for k in ("Kernel Name", "Metric Name", "Metric Value", "Metric Unit"))
    agg = collections.OrderedDict()
    for r in rows[1:]:
        if r[mi] != "gpu__time_duration.sum":
            continue
        name = r[ki].split("(")[0]
        a = agg.setdefault(name, [0, 0.0])
        a[0] += 1
        a[1] += float(r[vi].replace(",", "")) * SCALE[r[ui]]
    tot = sum(a[1] for a in agg.values())
    lines = ["| kernel | launches | total ms | share |", "|---|---|---|---|"]
    for k, (n, t) in sorted(agg.items(), key=lambda kv: -kv[1][1]):
        lines.append(f"| `{k}` | {n} | {t:.3f} | {100 * t / tot:.2f}% |")
    lines.append(f"| all | {sum(a[0] for a in agg.values())} | {tot:.3f} | 100% |")
    return "\n".join(lines)


if __name__ == "__main__":
    print(summarize(sys.argv[1]))
