"""The batched ensemble (GPU): every member of an ensemble step computes what ocean_step
computes for it alone (to rounding: the ensemble kernels are a second compiled instance of
the same kernel bodies, free to fuse multiply-adds differently), any launch shapes the
autotuner picks give bit-identical results, and the members follow the FP64 oracle."""
import numpy as np
import pytest

from paper_2309_06662_gb300 import inputs, ocean
from tests.parity import max_rel

FIELDS = ("u", "v", "T_anom", "S_anom", "eta", "Gu_prev", "GT_prev")
PRECISIONS = [pytest.param(ocean.OCEAN_MIXED, id="mixed"), pytest.param(ocean.OCEAN_FP64, id="fp64")]


def _cases(count=7, seed=40):
    # uneven sizes, including a member narrower than one tile and one region
    return inputs.ensemble_cases(count, seed=seed, n_lo=20, n_hi=90, levels=(4, 8, 12))


def _alone(cases, precision, steps):
    """The same members stepped one by one with ocean_step (own handles)."""
    out = []
    for c in cases:
        m = ocean.Ocean(c, precision=precision)
        m.step(steps)
        out.append({f: m.get(f) for f in FIELDS})
        m.close()
    return out


@pytest.mark.gpu
@pytest.mark.parametrize("precision", PRECISIONS)
def test_ensemble_step_is_each_member_alone(precision):
    cases = _cases()
    E = ocean.Ensemble(cases, precision=precision)
    E.step(6)                     # Euler start, then both graph parities
    ref = _alone(cases, precision, 6)
    tol = 1e-5 if precision == ocean.OCEAN_MIXED else 1e-13
    for i, m in enumerate(E.members):
        assert m.nstep == 6
        for f in FIELDS:
            assert max_rel(m.get(f), ref[i][f]) <= tol, (i, f)
    assert E.launches == 6 * (6 + 5)
    E.close()


@pytest.mark.gpu
def test_autotuned_shapes_keep_results_bitwise():
    cases = _cases(seed=41)
    E = ocean.Ensemble(cases)
    n = E.autotune(reps=1)
    assert n >= 1
    shapes = E.launch_shapes()
    for k, s in shapes.items():
        assert 1 <= s["grid"] <= max(1, s["items"]), (k, s)
    E.step(3)
    D = ocean.Ensemble(cases)     # default shapes, same kernels
    D.step(n + 3)
    for a, b in zip(E.members, D.members):
        for f in FIELDS:
            assert np.array_equal(a.get(f), b.get(f)), f
    E.close()
    D.close()


@pytest.mark.gpu
def test_members_follow_the_oracle():
    oracle = pytest.importorskip("oracle")
    cases = _cases(count=3, seed=42)
    E = ocean.Ensemble(cases, precision=ocean.OCEAN_FP64)
    E.step(10)
    for i, c in enumerate(cases):
        o = oracle.OracleModel(c)
        o.step(10)
        for f in ("u", "v", "T", "S", "eta"):
            assert max_rel(E.members[i].get(f), o.get(f)) <= 1e-10, (i, f)
    E.close()


@pytest.mark.gpu
def test_a_member_stepped_alone_puts_the_ensemble_out_of_step():
    cases = _cases(count=3, seed=43)
    E = ocean.Ensemble(cases)
    E.step(2)
    E.members[1].step(1)
    with pytest.raises(ocean.OceanError) as err:
        E.step(1)
    assert err.value.code == -6
    E.members[0].step(1)
    E.members[2].step(1)
    E.step(1)
    assert all(m.nstep == 4 for m in E.members)
    E.close()


@pytest.mark.gpu
def test_member_diagnostics_and_checkpoint():
    cases = _cases(count=3, seed=44)
    E = ocean.Ensemble(cases)
    d0 = [m.diagnostics() for m in E.members]
    E.step(4)
    for m, d in zip(E.members, d0):
        d1 = m.diagnostics()
        assert not d1["nonfinite"]
        # closed basins: tracer and volume conserved to roundoff of the FP32 state
        assert abs(d1["tracer_T"] - d["tracer_T"]) <= 1e-6 * abs(d["tracer_T"])
    # restart every member of a fresh ensemble from checkpoints: the continuation is
    # the same bit for bit
    cks = [m.checkpoint() for m in E.members]
    E.step(2)
    E2 = ocean.Ensemble(cases)
    for m, ck in zip(E2.members, cks):
        m.restore(ck)
    E2.step(2)
    for a, b in zip(E.members, E2.members):
        for f in FIELDS:
            assert np.array_equal(a.get(f), b.get(f)), f
    E.close()
    E2.close()


@pytest.mark.gpu
@pytest.mark.parametrize("precision", PRECISIONS)
def test_region_halo_widths_agree_to_rounding(precision):
    # the barotropic regions cut for 4 and 8 substeps per pass against the default 6: the
    # same sub-cycle, with the partial averages added into the accumulators at other
    # substeps (in FP64 the groupings differ only in the last bits)
    cases = _cases(count=5, seed=45)
    D = ocean.Ensemble(cases, precision=precision)
    assert D.region_substeps == 6
    D.step(6)
    tol = 1e-5 if precision == ocean.OCEAN_MIXED else 1e-13
    for bs in (4, 8):
        E = ocean.Ensemble(cases, precision=precision)
        E.region_substeps = bs
        assert E.region_substeps == bs
        E.step(6)
        assert E.launches == 6 * (6 + -(-30 // bs))
        for a, b in zip(E.members, D.members):
            for f in FIELDS:
                assert max_rel(a.get(f), b.get(f)) <= tol, (bs, f)
        E.close()
    D.close()


@pytest.mark.gpu
def test_region_autotuner_keeps_the_fastest_halo_width():
    cases = _cases(count=5, seed=46)
    E = ocean.Ensemble(cases)
    n = E.autotune_regions(reps=2)
    assert n == 6
    times = E.region_times()
    assert all(t > 0 for t in times.values()), times
    assert E.region_substeps == min(times, key=times.get)
    E.step(2)
    assert not any(m.diagnostics()["nonfinite"] for m in E.members)
    with pytest.raises(ocean.OceanError):
        E.region_substeps = 5
    E.close()
