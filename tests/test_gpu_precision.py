"""The mixed-precision form (FP32 fields and stencils; FP64 free surface, barotropic
averages and conservation sums) against FP64 references, field by field (GPU).

- 1/12 degree (4320 x 1680 x 48, the benchmark's workload), 200 steps: mixed against the
  FP64 GPU path on the whole grid (the oracle cannot step this grid).
- 1/2-degree restriction of the same recipe (720 x 280 x 48): mixed against the oracle.
- 1 degree (360 x 160 x 32): FP64 and mixed against the oracle, 100 steps.
Bars: relative L2 <= 2e-4 per prognostic field in the mixed form, max |gpu - oracle| /
max |oracle| <= 1e-10 in FP64.  The tracer anomalies T - T(0), S - S(0) are reported
beside the fields."""
import numpy as np
import pytest

from paper_2309_06662_gb300 import inputs, ocean
from tests.parity import STATE, field_error_table

pytestmark = pytest.mark.gpu

MIXED_TOL = 2e-4
FP64_TOL = 1e-10


def _wet(model):
    return model.get("T") != 0


def _snapshot(model):
    return {f: model.get(f) for f in STATE}


@pytest.mark.slow
def test_12th_degree_mixed_against_fp64_gpu_200_steps():
    case = inputs.latlon_12th_case()
    steps = case.steps
    m = ocean.Ocean(case, precision=ocean.OCEAN_MIXED)
    m.step(steps)
    assert not m.diagnostics()["nonfinite"]
    a = _snapshot(m)
    m.close()
    del m
    r = ocean.Ocean(case, precision=ocean.OCEAN_FP64)
    r.step(steps)
    b = _snapshot(r)
    r.close()
    del r
    wet = b["T"] != 0
    errs = field_error_table(a.get, b.get, wet, case.T, case.S)
    print("1/12 degree, mixed vs FP64 GPU, %d steps:" % steps, errs)
    for f in STATE:
        assert errs[f]["rel_l2"] <= MIXED_TOL, (f, errs[f])


@pytest.mark.slow
def test_half_degree_restriction_mixed_against_oracle():
    oracle = pytest.importorskip("oracle")
    case = inputs.latlon_half70_case()
    steps = 30
    g = ocean.Ocean(case, precision=ocean.OCEAN_MIXED)
    g.step(steps)
    o = oracle.OracleModel(case)
    o.step(steps)
    wet = _wet(o)
    errs = field_error_table(g.get, o.get, wet, case.T, case.S)
    print("1/2 degree, mixed vs oracle, %d steps:" % steps, errs)
    for f in STATE:
        assert errs[f]["rel_l2"] <= MIXED_TOL, (f, errs[f])


@pytest.mark.slow
def test_one_degree_fp64_and_mixed_against_oracle_100_steps():
    oracle = pytest.importorskip("oracle")
    case = inputs.latlon_1deg_case()
    steps = 100
    o = oracle.OracleModel(case)
    o.step(steps)
    wet = _wet(o)
    for prec in (ocean.OCEAN_FP64, ocean.OCEAN_MIXED):
        g = ocean.Ocean(case, precision=prec)
        g.step(steps)
        errs = field_error_table(g.get, o.get, wet, case.T, case.S)
        print("1 degree, %s vs oracle, %d steps:" % ("FP64" if prec == 0 else "mixed", steps), errs)
        for f in STATE:
            if prec == ocean.OCEAN_FP64:
                assert errs[f]["max_rel"] <= FP64_TOL, (f, errs[f])
            else:
                assert errs[f]["rel_l2"] <= MIXED_TOL, (f, errs[f])
        g.close()
