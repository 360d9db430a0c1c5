"""Writes tests/golden/box_oracle_diagnostics.txt by running the CPU oracle only.

The stored numbers are the oracle's own diagnostics of the seeded 32 x 32 x 8 box after
10 and 100 steps; the regression test re-runs the oracle and compares, so a change to
the oracle's arithmetic shows up as a diff of this file.
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2309_06662_gb300 import inputs  # noqa: E402

KEYS = ["tracer_T", "tracer_S", "volume_eta", "ke", "max_cfl"]


def compute():
    m = oracle.OracleModel(inputs.box_case())
    rows = []
    done = 0
    for n in (10, 100):
        m.step(n - done)
        done = n
        d = m.diagnostics()
        rows.append((n, [d[k] for k in KEYS]))
    return rows


if __name__ == "__main__":
    with open(os.path.join(HERE, "box_oracle_diagnostics.txt"), "w") as f:
        f.write("# oracle diagnostics of inputs.box_case() (seed 1); written by make_oracle_golden.py\n")
        f.write("# step " + " ".join(KEYS) + "\n")
        for n, vals in compute():
            f.write(f"{n} " + " ".join(repr(float(v)) for v in vals) + "\n")
