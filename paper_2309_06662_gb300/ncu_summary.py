"""Summarise an `ncu --metrics gpu__time_duration.sum --csv` launch list per kernel.

Usage: python -m paper_2309_06662_gb300.ncu_summary <launches.csv>
Prints, per kernel (template arguments folded), the launch count, total device time and
share of the captured total.  ncu times are cold-cache and serialised: compare shares.
"""
import collections
import csv
import re
import sys


def summarize(path):
    rows = list(csv.reader(open(path)))
    hdr, data = None, []
    for r in rows:
        if "Kernel Name" in r:
            hdr = r
            continue
        if hdr and len(r) == len(hdr):
            data.append(dict(zip(hdr, r)))
    scale = {"nsecond": 1.0, "usecond": 1e3, "msecond": 1e6, "second": 1e9}
    tot, cnt = collections.defaultdict(float), collections.Counter()
    for d in data:
        if d.get("Metric Name") != "gpu__time_duration.sum":
            continue
        m = re.search(r"\b(k_[A-Za-z0-9_]+)(<[^(]*>)?", d["Kernel Name"])
        name = (m.group(1) + (m.group(2) or "")) if m else d["Kernel Name"][:60]
        tot[name] += float(d["Metric Value"].replace(",", "")) * scale.get(d["Metric Unit"], 1.0)
        cnt[name] += 1
    total = sum(tot.values())
    out = [f"{'kernel':44s} {'launches':>8s} {'total_ms':>10s} {'share':>7s}"]
    for k, v in sorted(tot.items(), key=lambda x: -x[1]):
        out.append(f"{k:44s} {cnt[k]:8d} {v / 1e6:10.3f} {100 * v / total:6.2f}%")
    out.append(f"{'TOTAL':44s} {sum(cnt.values()):8d} {total / 1e6:10.3f}")
    return "\n".join(out)




KEY_METRICS = [
    "gpu__time_duration.sum", "launch__grid_size", "launch__block_size",
    "launch__registers_per_thread", "launch__occupancy_limit_registers",
    "launch__occupancy_limit_shared_mem", "dram__bytes_read.sum", "dram__bytes_write.sum",
    "gpu__dram_throughput.avg.pct_of_peak_sustained_elapsed",
    "sm__throughput.avg.pct_of_peak_sustained_elapsed",
    "sm__issue_active.avg.pct_of_peak_sustained_elapsed",
    "sm__warps_active.avg.pct_of_peak_sustained_active",
    "sm__inst_executed_pipe_alu.avg.pct_of_peak_sustained_active",
    "sm__pipe_fma_cycles_active.avg.pct_of_peak_sustained_active",
    "sm__inst_executed_pipe_lsu.avg.pct_of_peak_sustained_active",
    "sm__inst_executed_pipe_xu.avg.pct_of_peak_sustained_active",
    "sm__pipe_tensor_cycles_active.avg.pct_of_peak_sustained_active",
    "l1tex__data_bank_conflicts_pipe_lsu_mem_shared.sum",
    "lts__t_sector_hit_rate.pct",
]
STALL_PREFIX = "smsp__average_warps_issue_stalled_"


def raw_metrics(csv_text: str):
    """Key metrics of each launch in `ncu -i <rep> --page raw --csv` output."""
    rows = list(csv.reader(csv_text.splitlines()))
    hdr, units = rows[0], rows[1]
    out = []
    for r in rows[2:]:
        name = r[hdr.index("Kernel Name")] if "Kernel Name" in hdr else "?"
        m = re.search(r"\b(k_[A-Za-z0-9_]+)(<[^(]*>)?", name)
        lines = [f"kernel {m.group(0) if m else name[:60]}"]
        for k in KEY_METRICS:
            if k in hdr:
                i = hdr.index(k)
                lines.append(f"  {k:64s} {r[i]:>16s} {units[i]}")
        lines.append("  warp stalls per issued instruction (>= 0.1):")
        for i, k in enumerate(hdr):
            if k.startswith(STALL_PREFIX) and k.endswith("_per_issue_active.ratio"):
                try:
                    if float(r[i]) >= 0.1:
                        lines.append(f"    {k[len(STALL_PREFIX):-len('_per_issue_active.ratio')]:30s} {float(r[i]):6.2f}")
                except ValueError:
                    pass
        out.append("\n".join(lines))
    return "\n\n".join(out)


if __name__ == "__main__":
    if sys.argv[1] == "--raw":
        print(raw_metrics(sys.stdin.read()))
    else:
        print(summarize(sys.argv[1]))
