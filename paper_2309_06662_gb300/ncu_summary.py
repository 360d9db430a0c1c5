"""Summarise an `ncu --metrics gpu__time_duration.sum --csv` launch list per kernel.

Usage:
  python -m paper_2309_06662_gb300.ncu_summary <launches.csv>
      per kernel (template arguments folded): launch count, total device time and share
      of the captured total.  ncu times are cold-cache and serialised: compare shares.
  ncu -i <rep> --page raw --csv | python -m paper_2309_06662_gb300.ncu_summary --raw
      the key metrics and warp stalls of each captured launch.
  python -m paper_2309_06662_gb300.ncu_summary --traffic <dram.csv> <captured> <applied>
      DRAM bytes (read + write) per launch and per wet cell of the 3-D kernels from a
      capture of `dram__bytes_read.sum,dram__bytes_write.sum` on workload <captured>,
      printed as the "traffic_json:" line the benchmark reads for workload <applied>.
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


PHASE_OF = {"k_diag": "diag", "k_tracer": "tracer", "k_momentum": "momentum",
            "k_correct": "correct"}
BYTES = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}


def traffic(path, captured, applied):
    """Mean DRAM bytes per launch of each 3-D kernel, per wet cell of `captured`: these
    kernels touch each wet cell a fixed number of times, so the figure carries over to
    another grid of the same vertical structure by its wet-cell count."""
    import json
    from . import roofline
    from .inputs import WORKLOADS
    case = WORKLOADS[captured][0]()
    wet = roofline.wet_cells(case.depth, case.z_faces, case.params["min_depth"])
    rows = list(csv.reader(open(path)))
    hdr, per = None, collections.defaultdict(lambda: collections.defaultdict(float))
    for r in rows:
        if "Kernel Name" in r:
            hdr = r
            continue
        if not hdr or len(r) != len(hdr):
            continue
        d = dict(zip(hdr, r))
        m = re.search(r"\b(k_[A-Za-z0-9_]+)", d["Kernel Name"])
        if not m or m.group(1) not in PHASE_OF:
            continue
        key = (m.group(1), d["ID"])
        if d["Metric Name"] in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            per[key][d["Metric Name"]] += float(d["Metric Value"].replace(",", "")) * \
                BYTES.get(d["Metric Unit"], 1.0)
    sums, cnt = collections.defaultdict(float), collections.Counter()
    lines = [f"{'kernel':12s} {'launches':>8s} {'read_MB':>9s} {'write_MB':>9s} {'B/wet_cell':>10s}"]
    rd, wr = collections.defaultdict(float), collections.defaultdict(float)
    for (k, _), v in per.items():
        rd[k] += v["dram__bytes_read.sum"]
        wr[k] += v["dram__bytes_write.sum"]
        cnt[k] += 1
    for k in sorted(cnt, key=lambda x: list(PHASE_OF).index(x)):
        r_, w_ = rd[k] / cnt[k], wr[k] / cnt[k]
        sums[PHASE_OF[k]] = round((r_ + w_) / wet, 2)
        lines.append(f"{k:12s} {cnt[k]:8d} {r_ / 1e6:9.1f} {w_ / 1e6:9.1f} {sums[PHASE_OF[k]]:10.2f}")
    lines.append(f"wet cells of {WORKLOADS[captured][1]}: {wet}")
    lines.append("traffic_json: " + json.dumps({
        "workload": WORKLOADS[applied][1], "captured_on": WORKLOADS[captured][1],
        "source_digest": roofline.source_digest(), "bytes_per_wet_cell": dict(sums)}))
    return "\n".join(lines)


if __name__ == "__main__":
    if sys.argv[1] == "--traffic":
        print(traffic(*sys.argv[2:5]))
    elif sys.argv[1] == "--raw":
        print(raw_metrics(sys.stdin.read()))
    else:
        print(summarize(sys.argv[1]))
