"""Stored values: the paper's published SYPD figures and the oracle's own regression file."""
import os

import numpy as np

from paper_2309_06662_gb300 import inputs, metrics

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    with open(os.path.join(HERE, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def test_sypd_conversion_reproduces_paper_table():
    for run, dt, sps, sy, tol in _rows("paper_sypd.txt"):
        assert abs(metrics.sypd(float(dt), float(sps)) - float(sy)) <= float(tol), run


def test_oracle_regression_box_diagnostics():
    import oracle
    m = oracle.OracleModel(inputs.box_case())
    done = 0
    for row in _rows("box_oracle_diagnostics.txt"):
        n = int(row[0])
        m.step(n - done)
        done = n
        d = m.diagnostics()
        tT, tS, _vol, ke, cfl = (float(x) for x in row[1:])
        np.testing.assert_allclose([d["tracer_T"], d["tracer_S"], d["ke"], d["max_cfl"]],
                                   [tT, tS, ke, cfl], rtol=1e-9)
