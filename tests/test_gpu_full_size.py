"""The full 1/12-degree workload (4320 x 1680 x 48, as the benchmark runs it) against the
oracle on sampled columns (GPU).

The oracle cannot step the whole grid in seconds, but it can reproduce sampled columns
exactly: one step reaches at most N_s + 4 columns away (one column per barotropic
substep, plus the 3-D stencils), so a window of the full grid with walls 150 columns
from its centre gives, after two steps, the same centre block as the whole grid."""
import numpy as np
import pytest

from paper_2309_06662_gb300 import inputs, ocean
from tests.parity import max_rel, rel_l2

MARGIN = 150   # > 2 steps x (60 substeps + 4)
BLOCK = 5      # centre block compared: (2 BLOCK + 1)^2 columns
STEPS = 2


@pytest.fixture(scope="module")
def case():
    return inputs.latlon_12th_case()


def _samples(case):
    # away from the walls at the y ends; one near the equator, two at mid-latitudes
    return [(case.nx // 2, case.ny // 2), (700, 330), (3300, 1300)]


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [ocean.OCEAN_MIXED, ocean.OCEAN_FP64])
def test_sampled_columns_match_oracle_windows(case, precision):
    oracle = pytest.importorskip("oracle")
    g = ocean.Ocean(case, precision=precision)
    g.step(STEPS)
    assert not g.diagnostics()["nonfinite"]
    full = {f: g.get(f) for f in ("u", "v", "T", "S", "eta")}
    g.close()
    del g
    for (ic, jc) in _samples(case):
        i0, j0 = ic - MARGIN, jc - MARGIN
        w = 2 * MARGIN + 1
        win = inputs.latlon_window_case(case, i0, j0, w, w)
        o = oracle.OracleModel(win)
        o.step(STEPS)
        b = slice(MARGIN - BLOCK, MARGIN + BLOCK + 1)
        for f, a in full.items():
            ref = o.get(f)[..., b, b]
            got = a[..., jc - BLOCK:jc + BLOCK + 1, ic - BLOCK:ic + BLOCK + 1]
            if precision == ocean.OCEAN_FP64:
                assert max_rel(got, ref) <= 1e-10, (ic, jc, f)
            else:
                assert rel_l2(got, ref) <= 2e-4, (ic, jc, f)


@pytest.mark.gpu
@pytest.mark.slow
def test_time_step_300_s_is_past_the_explicit_limit_and_180_s_is_not(case):
    """The configured 1/12-degree step of 300 s is beyond the explicit internal-wave limit
    of the quasi-AB2 scheme next to 70 degrees (zonal spacing 3.2 km): the advective CFL
    number grows by orders of magnitude within 40 steps and the state turns non-finite
    (measured: CFL 0.013 after 5 steps, 0.64 after 30, 3.7 after 40, non-finite by 50).
    The paper's own 180 s stays healthy over the same span (CFL about 0.01)."""
    grown = {}
    for dt in (300.0, 180.0):
        m = ocean.Ocean(case.with_params(dt=dt), precision=ocean.OCEAN_MIXED)
        cfl, bad = [], False
        for _ in range(12):
            m.step(5)
            d = m.diagnostics()
            bad = bad or d["nonfinite"]
            cfl.append(d["max_cfl"])
            if bad:
                break
        grown[dt] = (bad, cfl)
        m.close()
        del m
    bad300, cfl300 = grown[300.0]
    assert bad300 or max(cfl300) > 1.0, cfl300
    bad180, cfl180 = grown[180.0]
    assert not bad180 and max(cfl180) < 0.05, cfl180
