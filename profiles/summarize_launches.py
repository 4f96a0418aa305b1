"""Summarise an ncu launch list (--metrics gpu__time_duration.sum --csv) per kernel.

Usage: python profiles/summarize_launches.py launches.csv
Prints launches, total device time and share per kernel name.  ncu times are
cold-cache and serialised: compare shares, not absolute times.
"""
import collections
import csv
import sys

SCALE = {"ns": 1e-3, "nsecond": 1e-3, "us": 1.0, "usecond": 1.0, "ms": 1e3, "msecond": 1e3, "s": 1e6, "second": 1e6}


def summarize(path):
    rows = list(csv.reader(open(path)))
    h = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
    hdr = rows[h]
    ki, vi, ui = hdr.index("Kernel Name"), hdr.index("Metric Value"), hdr.index("Metric Unit")
    tot, cnt = collections.defaultdict(float), collections.Counter()
    for r in rows[h + 1:]:
        if len(r) <= vi or not r[vi]:
            continue
        name = r[ki].split("(")[0].replace("sk::<unnamed>::", "").replace("void ", "")[:48]
        tot[name] += float(r[vi].replace(",", "")) * SCALE.get(r[ui], 1.0)
        cnt[name] += 1
    total = sum(tot.values())
    out = [f"{'kernel':48s} {'launches':>8s} {'total_us':>12s} {'share':>7s}"]
    for k, v in sorted(tot.items(), key=lambda x: -x[1]):
        out.append(f"{k:48s} {cnt[k]:8d} {v:12.1f} {100 * v / total:6.1f}%")
    return "\n".join(out)


if __name__ == "__main__":
    print(summarize(sys.argv[1]))
