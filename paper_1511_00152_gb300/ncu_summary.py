"""Summaries of Nsight Compute output for the profile notes.

  python -m paper_1511_00152_gb300.ncu_summary launches <launches.csv>
      per kernel: launches, total device time and share, from a launch list
      taken with --metrics gpu__time_duration.sum --csv (ncu times are
      cold-cache and serialised: compare shares, not absolute times);
  python -m paper_1511_00152_gb300.ncu_summary metrics <report.ncu-rep>
      the figures the notes quote for each captured launch (duration, DRAM
      bytes and throughput, shared-memory wavefronts and bank conflicts,
      pipe utilisation, occupancy, the largest warp-stall reasons).

Reads ncu's own output only; nothing here touches the GPU.
"""
import collections
import csv
import subprocess
import sys

SCALE = {"ns": 1e-3, "nsecond": 1e-3, "us": 1.0, "usecond": 1.0, "ms": 1e3, "msecond": 1e3,
         "s": 1e6, "second": 1e6}

METRICS = [
    "gpu__time_duration.sum", "dram__bytes_read.sum", "dram__bytes_write.sum",
    "gpu__dram_throughput.avg.pct_of_peak_sustained_elapsed",
    "sm__warps_active.avg.pct_of_peak_sustained_active",
    "smsp__issue_active.avg.pct_of_peak_sustained_active",
    "l1tex__throughput.avg.pct_of_peak_sustained_active",
    "l1tex__data_pipe_lsu_wavefronts_mem_shared.sum",
    "l1tex__data_bank_conflicts_pipe_lsu_mem_shared.sum",
    "sm__pipe_tensor_cycles_active.avg.pct_of_peak_sustained_active",
    "sm__inst_executed_pipe_fp64.avg.pct_of_peak_sustained_active",
    "sm__pipe_fma_cycles_active.avg.pct_of_peak_sustained_active",
    "launch__registers_per_thread", "launch__grid_size", "launch__block_size",
    "launch__shared_mem_per_block_dynamic",
]


def launches(path):
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


def metrics(report):
    raw = subprocess.run(["ncu", "-i", report, "--page", "raw", "--csv"], capture_output=True,
                         text=True, check=True).stdout
    rows = list(csv.reader(raw.splitlines()))
    hdr, units, data = rows[0], rows[1], rows[2:]
    out = []
    if "Kernel Name" in hdr:
        i = hdr.index("Kernel Name")
        out.append("launches: " + " | ".join(d[i].split("(")[0][-60:] for d in data))
    for w in METRICS:
        if w in hdr:
            i = hdr.index(w)
            out.append(f"{w:66s} {units[i][:10]:10s} " + " ".join(d[i] for d in data))
    stalls = [(h, i) for i, h in enumerate(hdr)
              if h.startswith("smsp__average_warps_issue_stalled")
              and h.endswith("_per_issue_active.ratio")]
    stalls.sort(key=lambda x: -float(data[0][x[1]] or 0))
    for h, i in stalls[:6]:
        out.append(f"stall {h[34:-len('_per_issue_active.ratio')]:40s} " +
                   " ".join(d[i] for d in data))
    return "\n".join(out)


if __name__ == "__main__":
    if len(sys.argv) != 3 or sys.argv[1] not in ("launches", "metrics"):
        sys.exit(__doc__)
    print(launches(sys.argv[2]) if sys.argv[1] == "launches" else metrics(sys.argv[2]))
