"""Host logic of bench.py on CPU: the max-over-ranks timing with a world-size-2 gloo
group, and the reference arm (the CPU oracle) on rank 0 only."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    q.put((rank, bench.max_over_ranks(1.5 + rank, dist), bench.max_over_ranks(7.0 - rank, dist)))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo_world_size_2():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 2000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert got == [(0, 2.5, 7.0), (1, 2.5, 7.0)]
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25) == 3.25        # no process group


def _bench(args, env_extra):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, env=env,
                          capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_line_on_rank_0():
    r = _bench(["--impl", "reference", "--workload", "box", "--steps", "2", "--warmup", "1"],
               {"RANK": "0", "WORLD_SIZE": "1", "OMP_NUM_THREADS": "2"})
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 2
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["config"]["workload"] == "box_32x32x8"


def test_reference_arm_other_ranks_do_no_work():
    r = _bench(["--impl", "reference", "--workload", "box", "--steps", "2", "--warmup", "1"],
               {"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr
    assert not [l for l in r.stdout.splitlines() if l.startswith("{")]


def test_traffic_summary_reads_ncu_csv_and_matches_the_code_digest(tmp_path):
    # the bench's DRAM-traffic figure comes from an ncu CSV summarised per wet cell and is
    # used only while the kernels' code digest matches the one recorded with it
    import csv
    sys.path.insert(0, ROOT)
    import bench
    from paper_2309_06662_gb300 import roofline
    hdr = ["ID", "Process ID", "Process Name", "Host Name", "Kernel Name", "Context",
           "Stream", "Block Size", "Grid Size", "Device", "CC", "Section Name",
           "Metric Name", "Metric Unit", "Metric Value"]
    path = tmp_path / "dram.csv"
    with open(path, "w", newline="") as f:
        w = csv.writer(f)
        w.writerow(["==PROF== profiler banner"])
        w.writerow(hdr)
        for lid, (k, rd, wr) in enumerate([("k_tracer<float, 1>", "2.0", "1.0"),
                                            ("k_tracer<float, 1>", "4.0", "1.0"),
                                            ("k_diag<float>", "1.0", "0.5"),
                                            ("k_diag_sums<float>", "9.0", "9.0")]):
            for name, unit, val in (("dram__bytes_read.sum", "Gbyte", rd),
                                    ("dram__bytes_write.sum", "Gbyte", wr),
                                    ("gpu__time_duration.sum", "ns", "1000")):
                w.writerow([str(lid), "1", "p", "h", "void <unnamed>::" + k + "(KP<T1>)", "1",
                            "13", "(32, 8, 1)", "(1, 1, 1)", "0", "10.3", "s", name, unit, val])
    out = bench.ncu_traffic(str(path), "box", "box")
    line = [l for l in out.splitlines() if l.startswith("traffic_json:")][0]
    d = json.loads(line.split(":", 1)[1])
    from paper_2309_06662_gb300 import inputs
    c = inputs.box_case()
    wet = roofline.wet_cells(c.depth, c.z_faces, c.params["min_depth"])
    # mean over launches of read + write, per wet cell; kernels outside the table skipped
    assert abs(d["bytes_per_wet_cell"]["tracer"] - round(4.0e9 / wet, 2)) < 0.01
    assert abs(d["bytes_per_wet_cell"]["diag"] - round(1.5e9 / wet, 2)) < 0.01
    assert set(d["bytes_per_wet_cell"]) == {"tracer", "diag"}
    assert d["source_digest"] == roofline.source_digest()
    tfile = tmp_path / "traffic.txt"
    tfile.write_text(out + "\n")
    assert roofline.load_traffic(str(tfile), d["workload"], roofline.source_digest()) == \
        d["bytes_per_wet_cell"]
    assert roofline.load_traffic(str(tfile), d["workload"], "0" * 16) is None


def test_code_digest_ignores_comments_and_layout(tmp_path):
    sys.path.insert(0, ROOT)
    from paper_2309_06662_gb300 import roofline
    src = tmp_path / "csrc"
    src.mkdir()
    body = "int f(int x) {\n    return x + 1;   // one more\n}\n/* block\n comment */\n"
    (src / "ocean_kernels.cu").write_text(body)
    (src / "ocean_internal.cuh").write_text("#define A 1\n")
    d0 = roofline.source_digest(str(src))
    (src / "ocean_kernels.cu").write_text("int f(int x)\n{ return x + 1; }  // reworded\n")
    assert roofline.source_digest(str(src)) == d0
    (src / "ocean_kernels.cu").write_text("int f(int x) { return x + 2; }\n")
    assert roofline.source_digest(str(src)) != d0
