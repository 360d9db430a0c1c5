#!/usr/bin/env python
"""Benchmark of one baroclinic time step of the hydrostatic free-surface ocean on GB300.

Workload (default): the 1/12-degree lat-lon configuration, 4320 x 1680 x 48 cells
(70S-70N), dt = 180 s, 60 barotropic substeps, in the mixed-precision form (FP32 fields
and stencils; FP64 free surface and conservation sums).
`--workload ensemble96` times the batched ensemble instead: 96 closed basins of seeded
uneven sizes (32-512 x 32-512 x 8-48), stepped together.  `--workload learned_half` times
the 1/2-degree step with the learned column closure (network 288-256-256-256-144 on every
column, seeded weights) and the closure's BF16 tensor-core GEMM chain.  Inputs are
seeded and synthetic: random-field bathymetry and stratified T/S with noise stand in for
the ECCO2-forced realistic domain of the paper (Sec. "How performance was measured").

Prints one JSON line.  `value` is whole-job cell-updates/s (grid cells, land included,
times steps, summed over ranks, over the max-over-ranks device time), state resident in
HBM.  The default run also measures every other configuration (`configs`: the 1-degree
grid in the mixed form and in FP64, the aqua-planet per-GPU workload of the paper's weak
scaling, the 96-basin ensemble against its members one by one, the learned closure
against the Richardson-number step) and the per-field difference of the mixed form from
the FP64 path (`errors`).  `e2e` is the same metric through the C ABI with host buffers: every step uploads
the surface wind stress from host memory and reads the diagnostics back.  `--impl
reference` times the CPU oracle instead, on a bounded window of the same workload.
"""
from __future__ import annotations

import argparse
import collections
import csv
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count() or 1))

import numpy as np  # noqa: E402

from paper_2309_06662_gb300 import inputs, metrics, roofline  # noqa: E402

WORKLOADS = inputs.WORKLOADS
FALLBACK_HBM_GBS = 6800.0


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def max_over_ranks(x: float, dist=None) -> float:
    """The largest value of x over the ranks of the process group (x itself without one);
    the tensor lives where the group's backend communicates (CUDA for NCCL, host for gloo)."""
    if dist is None:
        return x
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def measured_tensor_peak():
    """Dense BF16 tensor peak (TFLOP/s): the measured burst figure, else the fallback."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        if "bf16_tflops" in d:
            return float(d["bf16_tflops"]), "measured bf16_tflops (burst)"
    return 1900.0, "fallback 1.9 PFLOP/s bf16"


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.out = None

    def __enter__(self):
        try:
            self.out = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu)], stdout=self.out, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.out is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.out.flush()
        with open(self.out.name) as f:
            rows = [ln.strip().split(",") for ln in f if ln.strip()]
        os.unlink(self.out.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for n, val in zip(names, r[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- CPU oracle

def oracle_sample(case):
    """The bounded sample of the workload the CPU oracle runs: a 96 x 96 column window of
    a large lat-lon grid (walls at the window edges), or the whole grid when small."""
    if case.kind == 1 and case.nx >= 200:
        wx, wy = 96, 96
        i0, j0 = case.nx // 2, case.ny // 2
        desc = (f"{wx}x{wy}x{case.nz} window of the {case.nx}x{case.ny}x{case.nz} workload at "
                f"(i0={i0}, j0={j0}), walls at the window edges")
        return inputs.latlon_window_case(case, i0, j0, wx, wy), desc
    return case, f"the full {case.nx}x{case.ny}x{case.nz} workload"


def _time_oracle(m, seconds: float, steps_cap: int):
    t0 = time.perf_counter()
    n = 0
    while n < steps_cap:
        m.step(1)
        n += 1
        if time.perf_counter() - t0 >= seconds and n >= 2:
            break
    return n, time.perf_counter() - t0


def run_oracle_sample(case, seconds: float, warmup: int = 1, steps_cap: int = 10_000,
                      single_thread: bool = True):
    """Time the CPU oracle on the bounded sample for about `seconds` on all host cores
    (and, unless single_thread is False, for a third of that on one core); cell-updates/s."""
    import oracle
    sample, desc = oracle_sample(case)
    m = oracle.OracleModel(sample)
    m.step(warmup)   # the forward-Euler first step stays outside the timing
    cores = oracle.get_threads()
    n, dt = _time_oracle(m, seconds, steps_cap)
    cells = sample.nx * sample.ny * sample.nz
    out = {"value": cells * n / dt, "unit": "cell-updates/s", "kind": "oracle",
           "cores": cores,
           "sample": f"{desc}; {n} steps in {dt:.1f} s (plain FP64 C, OpenMP over rows)",
           "s_per_step": dt / n}
    if single_thread:
        oracle.set_threads(1)
        n1, dt1 = _time_oracle(m, seconds / 3, steps_cap)
        oracle.set_threads(cores)
        out["single_thread"] = {"value": cells * n1 / dt1, "cores": 1,
                                "sample": f"the same window, {n1} steps in {dt1:.1f} s on one core"}
    return out



# ----------------------------------------------------------------------------- ncu summaries
# Post-processing of ncu output into the short summaries kept under profiles/:
#   python bench.py --ncu-launches <launches.csv>
#   ncu -i <rep> --page raw --csv | python bench.py --ncu-raw
#   python bench.py --ncu-traffic <dram.csv> <captured workload> <applied workload>




def ncu_launches(path):
    """Per kernel (template arguments folded) of an `ncu --metrics gpu__time_duration.sum
    --csv` launch list: launches, total device time and share of the captured total
    (ncu times are cold-cache and serialised: compare shares)."""
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


NCU_KEY_METRICS = [
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
NCU_STALL_PREFIX = "smsp__average_warps_issue_stalled_"


def ncu_raw(csv_text: str):
    """Key metrics of each launch in `ncu -i <rep> --page raw --csv` output."""
    rows = list(csv.reader(csv_text.splitlines()))
    hdr, units = rows[0], rows[1]
    out = []
    for r in rows[2:]:
        name = r[hdr.index("Kernel Name")] if "Kernel Name" in hdr else "?"
        m = re.search(r"\b(k_[A-Za-z0-9_]+)(<[^(]*>)?", name)
        lines = [f"kernel {m.group(0) if m else name[:60]}"]
        for k in NCU_KEY_METRICS:
            if k in hdr:
                i = hdr.index(k)
                lines.append(f"  {k:64s} {r[i]:>16s} {units[i]}")
        lines.append("  warp stalls per issued instruction (>= 0.1):")
        for i, k in enumerate(hdr):
            if k.startswith(NCU_STALL_PREFIX) and k.endswith("_per_issue_active.ratio"):
                try:
                    if float(r[i]) >= 0.1:
                        lines.append(f"    {k[len(NCU_STALL_PREFIX):-len('_per_issue_active.ratio')]:30s} {float(r[i]):6.2f}")
                except ValueError:
                    pass
        out.append("\n".join(lines))
    return "\n\n".join(out)


NCU_PHASE_OF = {"k_diag": "diag", "k_tracer": "tracer", "k_momentum": "momentum",
            "k_correct": "correct"}
NCU_BYTES = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}


def ncu_traffic(path, captured, applied):
    """Mean DRAM bytes per launch of each 3-D kernel, per wet cell of `captured`: these
    kernels touch each wet cell a fixed number of times, so the figure carries over to
    another grid of the same vertical structure by its wet-cell count."""
    WORKLOADS = inputs.WORKLOADS
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
        if not m or m.group(1) not in NCU_PHASE_OF:
            continue
        key = (m.group(1), d["ID"])
        if d["Metric Name"] in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            per[key][d["Metric Name"]] += float(d["Metric Value"].replace(",", "")) * \
                NCU_BYTES.get(d["Metric Unit"], 1.0)
    sums, cnt = collections.defaultdict(float), collections.Counter()
    lines = [f"{'kernel':12s} {'launches':>8s} {'read_MB':>9s} {'write_MB':>9s} {'B/wet_cell':>10s}"]
    rd, wr = collections.defaultdict(float), collections.defaultdict(float)
    for (k, _), v in per.items():
        rd[k] += v["dram__bytes_read.sum"]
        wr[k] += v["dram__bytes_write.sum"]
        cnt[k] += 1
    for k in sorted(cnt, key=lambda x: list(NCU_PHASE_OF).index(x)):
        r_, w_ = rd[k] / cnt[k], wr[k] / cnt[k]
        sums[NCU_PHASE_OF[k]] = round((r_ + w_) / wet, 2)
        lines.append(f"{k:12s} {cnt[k]:8d} {r_ / 1e6:9.1f} {w_ / 1e6:9.1f} {sums[NCU_PHASE_OF[k]]:10.2f}")
    lines.append(f"wet cells of {WORKLOADS[captured][1]}: {wet}")
    lines.append("traffic_json: " + json.dumps({
        "workload": WORKLOADS[applied][1], "captured_on": WORKLOADS[captured][1],
        "source_digest": roofline.source_digest(), "bytes_per_wet_cell": dict(sums)}))
    return "\n".join(lines)


# ----------------------------------------------------------------------------- main

def parse():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="latlon_12th")
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--error-steps", type=int, default=20,
                    help="steps of the mixed-vs-FP64 comparison (0: skip)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the other configurations in the default run")
    return ap.parse_args()


def reference_arm(args, rank: int):
    """The oracle on the host cores, on the same workload's config, metric and unit: W
    untimed steps, then K timed steps of the bounded sample."""
    if rank != 0:
        return
    import oracle
    make, wname = WORKLOADS[args.workload]
    case = make()
    member = ""
    if isinstance(case, list):          # an ensemble: its first member stands in
        case, member = case[0], " (member 0 of the ensemble)"
    sample, desc = oracle_sample(case)
    desc += member
    m = oracle.OracleModel(sample)
    m.step(max(1, args.warmup))
    t0 = time.perf_counter()
    m.step(args.steps)
    dt = time.perf_counter() - t0
    value = sample.nx * sample.ny * sample.nz * args.steps / dt
    cores = int(os.environ.get("OMP_NUM_THREADS", "1"))
    line = {
        "impl": "reference", "metric": "cell_updates_per_s", "value": value,
        "unit": "cell-updates/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_block(case, wname, "FP64 (CPU oracle)"),
        "cpu_baseline": {"value": value, "unit": "cell-updates/s", "kind": "oracle",
                         "cores": cores,
                         "sample": f"{desc}; {args.steps} steps in {dt:.1f} s (plain FP64 C, "
                                   f"OpenMP over rows)"},
        "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def mixed_vs_fp64(case, steps: int):
    """Per-field difference of the mixed form from the FP64 path after `steps` steps from
    the same initial state (both on the GPU): relative L2 and max-relative over each field,
    and the relative L2 of the bulk (all but the 0.1% of cells with the largest difference:
    the convective branch of the closure flips in a few cells where FP32 rounding moves
    N^2 across zero, and those cells carry most of the squared difference)."""
    import torch
    from paper_2309_06662_gb300 import ocean
    fields = ("u", "v", "T", "S", "eta")
    snap = {}
    for prec in (ocean.OCEAN_MIXED, ocean.OCEAN_FP64):
        m = ocean.Ocean(case, precision=prec)
        m.step(steps)
        snap[prec] = {f: m.get(f) for f in fields}
        m.close()
        del m
        torch.cuda.empty_cache()
    out = {"steps": steps, "against": "FP64 GPU path (itself within 1e-10 of the oracle)"}
    for f in fields:
        a, r = snap[ocean.OCEAN_MIXED][f], snap[ocean.OCEAN_FP64][f]
        d = np.abs(a - r)
        nr = float(np.linalg.norm(r))
        flat = d.ravel()
        n = flat.size // 1000
        keep = np.argpartition(flat, flat.size - n)[: flat.size - n] if n else slice(None)
        out[f] = {"rel_l2": float(np.linalg.norm(d) / nr) if nr else 0.0,
                  "max_rel": float(d.max() / np.abs(r).max()) if np.abs(r).max() else 0.0,
                  "bulk_rel_l2": float(np.linalg.norm(flat[keep]) / np.linalg.norm(r.ravel()[keep]))}
    return out


def single_model(case, precision: int, steps: int, warmup: int, local: int, dist=None):
    """Device-resident timing of one model (CUDA events on its stream around `steps`
    graph-replayed steps after `warmup`), the per-phase times of up to 5 more steps, the
    roofline of the heaviest single-kernel phase and the clocks seen."""
    import torch
    from paper_2309_06662_gb300 import ocean
    p = case.params
    esz = 8 if precision == ocean.OCEAN_FP64 else 4
    wet = roofline.wet_cells(case.depth, case.z_faces, p["min_depth"])
    wet_cols = roofline.wet_columns(case.depth, p["min_depth"], case.z_faces)
    m = ocean.Ocean(case, precision=precision)
    m.step_async(max(1, warmup))
    m.sync()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = m.launches
    with ClockSampler(local) as clk:
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        ev0.record()
        m.step_async(steps)
        ev1.record()
        torch.cuda.synchronize()
    ms = max_over_ranks(ev0.elapsed_time(ev1) / steps, dist)
    launches = m.launches - l0
    m.profile(True)
    m.step_async(min(steps, 5))
    m.sync()
    phases, nprof = m.phase_times()
    m.profile(False)
    healthy = not m.diagnostics()["nonfinite"]
    m.close()
    del m
    torch.cuda.empty_cache()
    peak, peak_src = measured_peaks()
    fr = {}
    for k in roofline.KERNEL_WORDS:
        t = phases[k] / nprof
        gbs = roofline.KERNEL_WORDS[k] * esz * wet / (t / 1e3) / 1e9
        fr[k] = {"ms": round(t, 4), "GBs": round(gbs, 1), "frac": round(gbs / peak, 3)}
    tb = phases["barotropic"] / nprof
    bb = roofline.barotropic_bytes_per_column(esz, int(p["n_substeps"])) * wet_cols
    fr["barotropic"] = {"ms": round(tb, 4), "GBs": round(bb / (tb / 1e3) / 1e9, 1),
                        "frac": round(bb / (tb / 1e3) / 1e9 / peak, 3)}
    top = max(roofline.KERNEL_WORDS, key=lambda k: fr[k]["ms"])
    step_bytes = roofline.STEP_WORDS_PER_CELL * esz * wet + bb
    return {"value": metrics.cell_updates_per_s(case.nx, case.ny, case.nz, ms / 1e3),
            "unit": "cell-updates/s", "ms_per_step": ms, "steps": steps,
            "sypd": metrics.sypd(p["dt"], ms / 1e3), "dt_s": p["dt"],
            "roofline": {"bound": "hbm", "kernel": top, "frac": fr[top]["frac"],
                         "achieved": fr[top]["GBs"], "peak": peak, "unit": "GB/s",
                         "peak_source": f"{peak_src} hbm_gbs"},
            "step_hbm_frac": step_bytes / (ms / 1e3) / 1e9 / peak,
            "phases": fr, "gpu_launches": launches, "healthy": healthy,
            "clocks": clk.summary()}


def other_configs(args, rank, world, local, dist, case12=None):
    """Every other configuration of the benchmark, measured in the default run: the
    1/12-degree step with the optional vertical schemes (stretched-level WENO
    coefficients, WENO vertical momentum advection), the 1-degree grid in the mixed form
    and in FP64 side by side, the aqua-planet per-GPU workload of the paper's weak scaling
    (FP64 as the paper ran it, and mixed), the 96-basin ensemble against its members
    stepped one by one, and the 1/2-degree step with the learned closure against the
    Richardson-number step."""
    import torch
    from paper_2309_06662_gb300 import ocean
    out = {}
    if case12 is not None:
        vs = single_model(case12.with_params(vertical_weno=1, momentum_vadv=1), ocean.OCEAN_MIXED,
                          10, 3, local, dist)
        vs["schemes"] = "vertical_weno=STRETCHED, momentum_vadv=WENO"
        out["latlon_12th_vertical_weno"] = vs
    c1 = inputs.latlon_1deg_case()
    mixed = single_model(c1, ocean.OCEAN_MIXED, 50, 5, local, dist)
    fp64 = single_model(c1, ocean.OCEAN_FP64, 10, 2, local, dist)
    out["latlon_1deg_360x160x32"] = {"mixed": mixed, "fp64": fp64,
                                     "mixed_over_fp64": mixed["value"] / fp64["value"]}
    ap = inputs.aquaplanet_case()
    apf = single_model(ap, ocean.OCEAN_FP64, 5, 1, local, dist)
    apm = single_model(ap, ocean.OCEAN_MIXED, 20, 3, local, dist)
    out["aquaplanet_1/6deg_2160x900x100"] = {
        "fp64": apf, "mixed": apm, "mixed_over_fp64": apm["value"] / apf["value"],
        "paper_per_gpu_context": "3.4e8 cell-updates/s per A100 in FP64 (768 A100s, 2.1e11 cells, "
                                 "0.81 s per step; other hardware, context only)"}
    keep = lambda d, ks: {k: d[k] for k in ks if k in d}
    sub = argparse.Namespace(**vars(args))
    sub.steps, sub.warmup, sub.e2e_steps = 10, 3, 2
    ens = ensemble_main(sub, inputs.ensemble_cases(96, seed=5), "ensemble_96_basins", rank,
                        world, local, dist, with_cpu=False)
    torch.cuda.empty_cache()
    if ens is not None:
        out["ensemble_96_basins"] = keep(ens, ["value", "unit", "ms_per_step", "one_by_one",
                                               "roofline", "step_hbm", "e2e", "gpu_launches",
                                               "clocks", "config", "autotune"])
    lrn = learned_main(sub, inputs.latlon_half_case(), WORKLOADS["learned_half"][1], rank, world,
                       local, dist, with_cpu=False)
    torch.cuda.empty_cache()
    if lrn is not None:
        out["learned_half_720x320x48"] = keep(lrn, ["value", "unit", "ms_per_step", "sypd",
                                                    "richardson_only", "roofline", "e2e",
                                                    "gpu_launches", "clocks", "healthy", "config"])
    return out


def config_block(case, wname, precision):
    p = case.params
    return {"workload": wname, "nx": case.nx, "ny": case.ny, "nz": case.nz,
            "cells": case.cells, "dt_s": p["dt"], "n_substeps": int(p["n_substeps"]),
            "precision": precision, "parallelism": "replicas (one full model per GPU)",
            "l2": "inputs larger than L2 (every 3-D field > 1 GB)"}


def learned_main(args, case, wname, rank, world, local, dist, with_cpu=True):
    """The 1/2-degree step with the learned closure in the loop (seeded network, feature
    statistics of the initial state), against the same step with the Richardson-number
    closure alone; the closure network's GEMM chain timed on all columns."""
    import torch
    from paper_2309_06662_gb300 import ocean

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    nz, H = case.nz, 256
    dims = [6 * nz, H, H, H, 3 * nz]
    params = inputs.mlp_seeded_params(11, dims, gain=0.5)
    sc = dict(kappa=1e-4, gT=1e-10, gS=1e-11, sFT=1.0, sFS=1.0, sGT=1.0, sGS=1.0)
    cells = case.nx * case.ny * case.nz
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    res = {}
    for name, closure in (("learned", ocean.OCEAN_CLOSURE_LEARNED), ("richardson", ocean.OCEAN_CLOSURE_RI)):
        m = ocean.Ocean(case, precision=ocean.OCEAN_MIXED, closure=closure,
                        closure_hidden=H if closure == ocean.OCEAN_CLOSURE_LEARNED else 0)
        if closure == ocean.OCEAN_CLOSURE_LEARNED:
            # feature statistics of the initial state over the entries that count (a
            # flat feature gets sigma 1), as the training pipeline computes them
            from paper_2309_06662_gb300 import closure_train
            mu, sd = closure_train.feature_stats(m.closure_features(np.zeros(6 * nz), np.ones(6 * nz)))
            m.set_closure(params, mu, sd, sc)
        m.step_async(args.warmup)
        m.sync()
        barrier()
        l0 = m.launches
        with ClockSampler(local) as clk:
            barrier()
            ev0.record()
            m.step_async(args.steps)
            ev1.record()
            barrier()
        res[name] = dict(ms=ev0.elapsed_time(ev1) / args.steps, launches=m.launches - l0,
                         clocks=clk.summary(), healthy=not m.diagnostics()["nonfinite"])
        if closure == ocean.OCEAN_CLOSURE_LEARNED:
            # end to end through the C ABI, per step: the wind stress from pinned host
            # memory, one step with the network in the loop, the diagnostics back
            taux = torch.from_numpy(np.ascontiguousarray(case.taux, dtype=np.float32)).pin_memory().numpy()
            tauy = torch.from_numpy(np.ascontiguousarray(case.tauy, dtype=np.float32)).pin_memory().numpy()
            barrier()
            t0 = time.perf_counter()
            for _ in range(args.e2e_steps):
                m.set_wind_stress(taux, tauy)
                m.step_async(1)
                d = m.diagnostics()
            barrier()
            e2e_s = max_over_ranks((time.perf_counter() - t0) / args.e2e_steps, dist)
            res[name]["e2e"] = {"value": cells / e2e_s * world, "unit": "cell-updates/s",
                                "h2d_bytes_per_step": int(taux.nbytes + tauy.nbytes),
                                "d2h_bytes_per_step": 8 * 8, "healthy": not d["nonfinite"],
                                "what": "per step: wind stress (FP32) host->device, one step "
                                        "with the network, diagnostics device->host"}
        m.close()
        del m
        torch.cuda.empty_cache()
    # the network's GEMM chain over all columns from BF16 features, as in the step:
    # 4 tcgen05 GEMMs with their fused epilogues
    M = case.nx * case.ny
    net = ocean.MLP(nz, H, M + (-M) % 8, params)
    Xc = torch.randn(M, 6 * nz, device="cuda").to(torch.bfloat16)
    for _ in range(3):
        net.forward_bf16(Xc)
    barrier()
    reps = 20
    ev0.record()
    for _ in range(reps):
        net.forward_bf16(Xc)
    ev1.record()
    barrier()
    ms_net = ev0.elapsed_time(ev1) / reps
    net.close()
    flops = 2.0 * M * sum(a * b for a, b in zip(dims[:-1], dims[1:]))
    peak, src = measured_tensor_peak()
    achieved = flops / (ms_net / 1e3) / 1e12
    ms = max_over_ranks(res["learned"]["ms"], dist)
    p = case.params
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and with_cpu:
        cpu = run_oracle_sample(case, args.cpu_seconds)
        cpu.pop("s_per_step", None)
        cpu["sample"] += " (Richardson-number closure: the oracle of the learned step is numpy, see oracle/closure.py)"
    if rank == 0:
        line = {
            "metric": "cell_updates_per_s", "value": cells / (ms / 1e3) * world,
            "unit": "cell-updates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+bf16",
            "data": "synthetic (seeded random-field bathymetry, stratified T/S; seeded network weights)",
            "config": {"workload": wname, "nx": case.nx, "ny": case.ny, "nz": case.nz,
                       "cells": cells, "dt_s": p["dt"], "n_substeps": int(p["n_substeps"]),
                       "precision": "mixed + BF16 closure network", "network": dims,
                       "parallelism": "replicas (one full model per GPU)",
                       "l2": "inputs larger than L2"},
            "sypd": metrics.sypd(p["dt"], ms / 1e3),
            "richardson_only": {"ms_per_step": res["richardson"]["ms"],
                                "closure_overhead_ms": ms - res["richardson"]["ms"]},
            "roofline": {"bound": "tensor", "kernel": "k_mlp_fused (whole network per 128-column tile)",
                         "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None,
                         "algorithmic_flops_per_chain": flops, "ms_per_chain": ms_net,
                         "peak_source": src},
            "e2e": res["learned"]["e2e"],
            "gpu_launches": res["learned"]["launches"],
            "clocks": res["learned"]["clocks"],
            "healthy": res["learned"]["healthy"],
            "cpu_baseline": cpu,
        }
        return line
    return None


def ensemble_main(args, cases, wname, rank, world, local, dist, with_cpu=True):
    """The batched ensemble: all members advanced by one graph launch per step, against
    the same members stepped one after another with ocean_step."""
    import torch
    from paper_2309_06662_gb300 import ocean

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    cells = sum(c.nx * c.ny * c.nz for c in cases)
    wet = sum(roofline.wet_cells(c.depth, c.z_faces, c.params["min_depth"]) for c in cases)
    wet_cols = sum(roofline.wet_columns(c.depth, c.params["min_depth"], c.z_faces) for c in cases)
    E = ocean.Ensemble(cases)
    stream = torch.cuda.ExternalStream(E.stream)
    # real steps, part of the warm-up: the barotropic region shape, then the launch shapes
    tuned = E.autotune_regions(reps=1)
    tuned += E.autotune(reps=2)
    E.step(max(1, args.warmup))
    barrier()
    launches0 = E.launches
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        ev0.record(stream)
        E.step_async(args.steps)
        ev1.record(stream)
        barrier()
    ms = ev0.elapsed_time(ev1) / args.steps
    launches = E.launches - launches0
    # the same members stepped one by one (single-model kernels, launches per member)
    ev0.record(stream)
    for m in E.members:
        m.step_async(1)
    ev1.record(stream)
    barrier()
    ms_seq = ev0.elapsed_time(ev1)
    ms_all = max_over_ranks(ms, dist)
    value = cells / (ms_all / 1e3) * world
    kinds = E.kind_times()
    esz = 4
    words = {"diag": roofline.KERNEL_WORDS["diag"], "tracer": roofline.KERNEL_WORDS["tracer"],
             "momentum": roofline.KERNEL_WORDS["momentum"],
             "correct": roofline.KERNEL_WORDS["correct"]}
    top = max(words, key=lambda k: kinds[k])
    peak, peak_src = measured_peaks()
    algo = words[top] * esz * wet
    achieved = algo / (kinds[top] / 1e3) / 1e9
    step_bytes = roofline.STEP_WORDS_PER_CELL * esz * wet + \
        roofline.barotropic_bytes_per_column(esz, 30) * wet_cols
    # end to end: per step every member's wind stress from pinned host memory, the
    # ensemble step, and every member's diagnostics read back
    winds = [(torch.from_numpy(np.ascontiguousarray(c.taux, dtype=np.float32)).pin_memory().numpy(),
              torch.from_numpy(np.ascontiguousarray(c.tauy, dtype=np.float32)).pin_memory().numpy())
             for c in cases]
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        for m, (tx, ty) in zip(E.members, winds):
            m.set_wind_stress(tx, ty)
        E.step_async(1)
        diags = [m.diagnostics() for m in E.members]
    barrier()
    e2e_s = (time.perf_counter() - t0) / args.e2e_steps
    healthy = all(not d["nonfinite"] and d["max_cfl"] < 1.0 for d in diags)
    shapes = E.launch_shapes()
    region_bs, region_ms = E.region_substeps, E.region_times()
    E.close()
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and with_cpu:
        cpu = run_oracle_sample(cases[0], args.cpu_seconds)
        cpu.pop("s_per_step", None)
        cpu["sample"] += " (member 0 of the ensemble)"
    if rank == 0:
        nz = sorted({c.nz for c in cases})
        line = {
            "metric": "cell_updates_per_s", "value": value, "unit": "cell-updates/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_all,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded closed beta-plane basins: random-field bathymetry, "
                    "stratified T/S with noise, zonal wind 0.05-0.2 N/m^2)",
            "config": {"workload": wname, "members": len(cases), "cells": cells,
                       "nx_range": [min(c.nx for c in cases), max(c.nx for c in cases)],
                       "ny_range": [min(c.ny for c in cases), max(c.ny for c in cases)],
                       "nz": nz, "dt_s": 600.0, "n_substeps": 30,
                       "precision": "mixed", "parallelism": "replicas (one ensemble per GPU)",
                       "l2": "inputs larger than L2 (the ensemble's state is ~10 GB)"},
            "wet_cells": wet,
            "one_by_one": {"ms_per_step": ms_seq, "value": cells / (ms_seq / 1e3),
                           "ensemble_speedup": ms_seq / ms},
            "autotune": {"steps": tuned, "shapes": shapes,
                         "kind_ms": {k: round(v, 4) for k, v in kinds.items()},
                         "region_substeps": region_bs,
                         "region_pass_ms": {str(k): round(v, 4) for k, v in region_ms.items()}},
            "step_hbm": {"algorithmic_bytes": step_bytes,
                         "GBs": step_bytes / (ms_all / 1e3) / 1e9,
                         "frac": step_bytes / (ms_all / 1e3) / 1e9 / peak, "of": peak_src},
            "roofline": {"bound": "hbm", "kernel": "k_ens_" + top, "achieved": achieved,
                         "peak": peak, "unit": "GB/s", "frac": achieved / peak, "traffic": None,
                         "algorithmic_bytes_per_launch": algo, "ms_per_launch": kinds[top],
                         "peak_source": f"{peak_src} hbm_gbs"},
            "e2e": {"value": cells / e2e_s, "unit": "cell-updates/s",
                    "h2d_bytes_per_step": int(sum(a.nbytes + b.nbytes for a, b in winds)),
                    "d2h_bytes_per_step": 64 * len(cases), "healthy": healthy,
                    "what": "per step: every member's wind stress host->device, one ensemble "
                            "step, every member's diagnostics device->host"},
            "gpu_launches": launches,
            "clocks": clk.summary(),
            "cpu_baseline": cpu,
        }
        return line
    return None


def ncu_cli(argv) -> bool:
    """The ncu post-processing modes; True when one of them ran."""
    if len(argv) >= 2 and argv[0] == "--ncu-launches":
        print(ncu_launches(argv[1]))
    elif argv and argv[0] == "--ncu-raw":
        print(ncu_raw(sys.stdin.read()))
    elif len(argv) >= 4 and argv[0] == "--ncu-traffic":
        print(ncu_traffic(*argv[1:4]))
    else:
        return False
    return True


def main():
    if ncu_cli(sys.argv[1:]):
        return
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        reference_arm(args, rank)
        return

    import torch
    from paper_2309_06662_gb300 import ocean

    torch.cuda.set_device(local)
    # a stream of our own: the library captures each step as a CUDA graph, which the
    # legacy default stream does not allow
    torch.cuda.set_stream(torch.cuda.Stream())
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    make, wname = WORKLOADS[args.workload]
    if args.workload in ("ensemble96", "learned_half"):
        fn = ensemble_main if args.workload == "ensemble96" else learned_main
        line = fn(args, make(), wname, rank, world, local, dist)
        if line is not None:
            print(json.dumps(line), flush=True)
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return
    case = make()
    p = case.params
    wet = roofline.wet_cells(case.depth, case.z_faces, p["min_depth"])
    wet_cols = roofline.wet_columns(case.depth, p["min_depth"], case.z_faces)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # ---------------------------------------------------------------- mixed, device-resident
    m = ocean.Ocean(case, precision=ocean.OCEAN_MIXED)
    m.step_async(args.warmup)
    m.sync()
    barrier()
    launches0 = m.launches
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        ev0.record()
        m.step_async(args.steps)
        ev1.record()
        barrier()
    ms = ev0.elapsed_time(ev1) / args.steps
    launches = m.launches - launches0
    # per-phase device times from the library's own events, on extra steps launched
    # without the step graph (the events sit between the phases)
    m.profile(True)
    m.step_async(min(args.steps, 5))
    m.sync()
    phases, nprof = m.phase_times()
    m.profile(False)
    ms_all = max_over_ranks(ms, dist)
    value = metrics.cell_updates_per_s(case.nx, case.ny, case.nz, ms_all / 1e3, replicas=world)

    # ---------------------------------------------------------------- roofline of the top kernel
    peak, peak_src = measured_peaks()
    esz = 4
    single = {k: phases[k] / nprof for k in roofline.KERNEL_WORDS}
    top = max(single, key=single.get)
    top_ms = single[top]
    algo = roofline.KERNEL_WORDS[top] * esz * wet
    achieved = algo / (top_ms / 1e3) / 1e9
    traffic = roofline.load_traffic(os.path.join(ROOT, "profiles", "traffic.txt"), wname,
                                    roofline.source_digest())
    tr = traffic.get(top) * wet if traffic and top in traffic else None
    step_bytes = roofline.STEP_WORDS_PER_CELL * esz * wet + \
        roofline.barotropic_bytes_per_column(esz, int(p["n_substeps"])) * wet_cols
    phase_frac = {}
    for k in roofline.KERNEL_WORDS:
        t = phases[k] / nprof
        phase_frac[k] = {"ms": round(t, 4),
                         "GBs": round(roofline.KERNEL_WORDS[k] * esz * wet / (t / 1e3) / 1e9, 1),
                         "frac": round(roofline.KERNEL_WORDS[k] * esz * wet / (t / 1e3) / 1e9 / peak, 3)}
    tb = phases["barotropic"] / nprof
    bb = roofline.barotropic_bytes_per_column(esz, int(p["n_substeps"])) * wet_cols
    phase_frac["barotropic"] = {"ms": round(tb, 4), "GBs": round(bb / (tb / 1e3) / 1e9, 1),
                                "frac": round(bb / (tb / 1e3) / 1e9 / peak, 3),
                                "kernels": -(-int(p["n_substeps"]) // 6) + 2}

    # ---------------------------------------------------------------- end to end, host buffers
    # the mixed model takes its wind in FP32 (ocean_set_wind_stress_f32: half the bytes)
    taux = torch.from_numpy(np.ascontiguousarray(case.taux, dtype=np.float32)).pin_memory().numpy()
    tauy = torch.from_numpy(np.ascontiguousarray(case.tauy, dtype=np.float32)).pin_memory().numpy()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        m.set_wind_stress(taux, tauy)
        m.step_async(1)
        d = m.diagnostics()
    barrier()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / args.e2e_steps, dist)
    e2e_value = metrics.cell_updates_per_s(case.nx, case.ny, case.nz, e2e_s, replicas=world)
    healthy = not d["nonfinite"] and d["max_cfl"] < 1.0
    m.close()
    del m
    torch.cuda.empty_cache()

    # ---------------------------------------------------------------- plain FP64 path
    fp64 = None
    if args.fp64_steps > 0:
        m64 = ocean.Ocean(case, precision=ocean.OCEAN_FP64)
        m64.step_async(1)
        m64.sync()
        barrier()
        ev0.record()
        m64.step_async(args.fp64_steps)
        ev1.record()
        barrier()
        ms64 = ev0.elapsed_time(ev1) / args.fp64_steps
        m64.close()
        del m64
        torch.cuda.empty_cache()
        v64 = metrics.cell_updates_per_s(case.nx, case.ny, case.nz, ms64 / 1e3, replicas=world)
        fp64 = {"value": v64, "ms_per_step": ms64, "steps": args.fp64_steps,
                "mixed_over_fp64": value / v64}

    errors = mixed_vs_fp64(case, args.error_steps) if rank == 0 and args.error_steps > 0 else None
    configs = None
    if args.workload == "latlon_12th" and not args.no_configs:
        configs = other_configs(args, rank, world, local, dist, case12=case)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = run_oracle_sample(case, args.cpu_seconds)
        cpu.pop("s_per_step", None)

    if rank == 0:
        line = {
            "metric": "cell_updates_per_s", "value": value, "unit": "cell-updates/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_all,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded random-field bathymetry, stratified T/S with noise, "
                    "zonal wind 0.1 cos(3 lat); stands in for the ECCO2-forced domains)",
            "config": config_block(case, wname, "mixed (FP32 fields and stencils; FP64 free "
                                                 "surface and sums)"),
            "sypd": metrics.sypd(p["dt"], ms_all / 1e3),
            "sim_days_per_day": metrics.sim_days_per_day(p["dt"], ms_all / 1e3),
            "wet_cells": wet,
            "step_hbm": {"algorithmic_bytes": step_bytes,
                         "GBs": step_bytes / (ms_all / 1e3) / 1e9,
                         "frac": step_bytes / (ms_all / 1e3) / 1e9 / peak,
                         "of": peak_src},
            "roofline": {"bound": "hbm", "kernel": top, "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak, "traffic": tr,
                         "algorithmic_bytes_per_launch": algo, "ms_per_launch": top_ms,
                         "peak_source": f"{peak_src} hbm_gbs"},
            "phases": phase_frac,
            "fp64": fp64,
            "errors": errors,
            "configs": configs,
            "e2e": {"value": e2e_value, "unit": "cell-updates/s",
                    "h2d_bytes_per_step": int(taux.nbytes + tauy.nbytes),
                    "d2h_bytes_per_step": 8 * 8, "healthy": healthy,
                    "what": "per step: wind stress (FP32) host->device, one step, diagnostics "
                            "(conservation sums, CFL, NaN check) device->host"},
            "gpu_launches": launches,
            "clocks": clk.summary(),
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
