"""Per-field error table of the mixed-precision form (and of the FP64 path) against FP64
references, at the configured sizes and step counts (needs a GPU; several minutes of
oracle time).  Test infrastructure: prints one JSON line per comparison.

    python tests/precision_report.py [--steps-half 200] [--steps-one 1000] [--steps-12th 200]
"""
import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2309_06662_gb300 import inputs, ocean  # noqa: E402
from tests.parity import STATE, field_error_table  # noqa: E402


def _round(d):
    return {k: ({kk: float("%.3g" % vv) for kk, vv in v.items()} if isinstance(v, dict) else v)
            for k, v in d.items()}


def snapshot(model):
    return {f: model.get(f) for f in STATE}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps-12th", type=int, default=200)
    ap.add_argument("--steps-half", type=int, default=200)
    ap.add_argument("--steps-one", type=int, default=1000)
    a = ap.parse_args()
    if a.steps_12th:
        case = inputs.latlon_12th_case()
        snaps = {}
        for prec in (ocean.OCEAN_MIXED, ocean.OCEAN_FP64):
            m = ocean.Ocean(case, precision=prec)
            m.step(a.steps_12th)
            snaps[prec] = snapshot(m)
            m.close()
            del m
        wet = snaps[ocean.OCEAN_FP64]["T"] != 0
        errs = field_error_table(snaps[ocean.OCEAN_MIXED].get, snaps[ocean.OCEAN_FP64].get, wet, case.T, case.S)
        print(json.dumps({"config": "1/12 degree 4320x1680x48", "steps": a.steps_12th,
                          "compare": "mixed vs FP64 GPU", "errors": _round(errs)}), flush=True)
    for name, make, steps in (("1/2 degree restriction 720x280x48", inputs.latlon_half70_case, a.steps_half),
                              ("1 degree 360x160x32", inputs.latlon_1deg_case, a.steps_one)):
        if not steps:
            continue
        case = make()
        o = oracle.OracleModel(case)
        o.step(steps)
        wet = o.get("T") != 0
        for prec, label in ((ocean.OCEAN_MIXED, "mixed"), (ocean.OCEAN_FP64, "FP64")):
            g = ocean.Ocean(case, precision=prec)
            g.step(steps)
            errs = field_error_table(g.get, o.get, wet, case.T, case.S)
            print(json.dumps({"config": name, "steps": steps, "compare": label + " vs oracle",
                              "errors": _round(errs)}), flush=True)
            g.close()


if __name__ == "__main__":
    main()
