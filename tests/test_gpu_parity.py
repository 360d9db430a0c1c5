"""CUDA path vs CPU oracle, element by element, on seeded inputs (needs a GPU).

FP64: max |gpu - oracle| / max |oracle| <= 1e-10 per prognostic field after the stated
number of steps.  Mixed precision (FP32 fields and stencils): relative L2 <= 2e-4.
"""
import numpy as np
import pytest

import oracle
from paper_2309_06662_gb300 import inputs, ocean
from tests.oracle_cases import NO_MIXING, flat_box, lake_at_rest, seeded_velocity
from tests.parity import max_rel, rel_l2, run_pair, state_errors

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
MIXED_TOL = 2e-4
DIAG = ["w", "p", "kappa", "nu", "Gu", "Gv", "GT", "GS"]


def _moving_state(case, seed=3, amp=0.05):
    case.u, case.v = seeded_velocity(case, seed, amp)
    return case


@pytest.mark.parametrize("make", [lambda: inputs.box_case(),
                                  lambda: _moving_state(inputs.latlon_small_case())])
def test_tendencies_and_diagnostics_fp64(make):
    c = make()
    g, o = run_pair(c, ocean.OCEAN_FP64, 0)
    g.tendencies()
    o.tendencies()
    for f in DIAG:
        err = max_rel(g.get(f), o.get(f))
        assert err < 1e-12, (f, err)


def test_box_fp64_100_steps():
    c = inputs.box_case()
    g, o = run_pair(c, ocean.OCEAN_FP64, 100)
    errs = state_errors(g, o)
    assert all(e <= FP64_TOL for e in errs.values()), errs
    assert g.nstep == 100


def test_latlon_small_fp64_50_steps():
    c = _moving_state(inputs.latlon_small_case())
    g, o = run_pair(c, ocean.OCEAN_FP64, 50)
    errs = state_errors(g, o)
    assert all(e <= FP64_TOL for e in errs.values()), errs


def test_box_mixed_100_steps():
    c = inputs.box_case()
    g, o = run_pair(c, ocean.OCEAN_MIXED, 100)
    errs = state_errors(g, o, rel_l2)
    assert all(e <= MIXED_TOL for e in errs.values()), errs
    # anomalies: the mean of T must not hide errors
    Ti = np.asarray(c.T)
    mask = o.get("T") != 0
    assert rel_l2((g.get("T") - Ti)[mask], (o.get("T") - Ti)[mask]) <= MIXED_TOL


def test_latlon_small_mixed_50_steps():
    c = _moving_state(inputs.latlon_small_case())
    g, o = run_pair(c, ocean.OCEAN_MIXED, 50)
    errs = state_errors(g, o, rel_l2)
    assert all(e <= MIXED_TOL for e in errs.values()), errs
    Ti = np.asarray(c.T)
    mask = o.get("T") != 0
    assert rel_l2((g.get("T") - Ti)[mask], (o.get("T") - Ti)[mask]) <= MIXED_TOL


@pytest.mark.parametrize("precision", [ocean.OCEAN_FP64, ocean.OCEAN_MIXED])
def test_aquaplanet_recipe_matches_oracle(precision):
    # the aqua-planet geometry (two ridges dividing the ocean into two basins that meet
    # south of 35S, 75S-75N) at 5 degrees: the periodic wrap through the ridges
    c = inputs.aquaplanet_case(nx=72, ny=30, nz=10, dt=1800.0, n_substeps=20)
    assert (c.depth == 0).any()
    g, o = run_pair(c, precision, 20)
    if precision == ocean.OCEAN_FP64:
        errs = state_errors(g, o)
        assert all(e <= FP64_TOL for e in errs.values()), errs
    else:
        errs = state_errors(g, o, rel_l2)
        assert all(e <= MIXED_TOL for e in errs.values()), errs


@pytest.mark.parametrize("precision", [ocean.OCEAN_FP64, ocean.OCEAN_MIXED])
def test_power_law_filter_matches_oracle(precision):
    # the sub-cycle averaged with the power-law weights (substep from their first moment)
    for c, steps in ((inputs.box_case().with_params(baro_filter=1), 60),
                     (_moving_state(inputs.latlon_small_case()).with_params(baro_filter=1), 30)):
        g, o = run_pair(c, precision, steps)
        if precision == ocean.OCEAN_FP64:
            errs = state_errors(g, o)
            assert all(e <= FP64_TOL for e in errs.values()), (c.name, errs)
        else:
            errs = state_errors(g, o, rel_l2)
            assert all(e <= MIXED_TOL for e in errs.values()), (c.name, errs)
        # and the filter changed the answer: the equal-weight run differs in eta
        b = oracle.OracleModel(c.with_params(baro_filter=0))
        b.step(steps)
        assert max_rel(b.get("eta"), o.get("eta")) > 1e3 * FP64_TOL


VERTICAL_SCHEMES = [dict(vertical_weno=1, momentum_vadv=0), dict(vertical_weno=0, momentum_vadv=1),
                    dict(vertical_weno=1, momentum_vadv=1)]


@pytest.mark.parametrize("scheme", VERTICAL_SCHEMES)
def test_vertical_schemes_tendencies_fp64(scheme):
    # stretched levels (5000 m in 12 levels, 40 m to 1270 m thick): the stretched-level
    # vertical WENO coefficients and the WENO flux form of the vertical momentum advection
    c = _moving_state(inputs.latlon_small_case()).with_params(**scheme)
    g, o = run_pair(c, ocean.OCEAN_FP64, 0)
    g.tendencies()
    o.tendencies()
    for f in ("Gu", "Gv", "GT", "GS"):
        err = max_rel(g.get(f), o.get(f))
        assert err < 1e-12, (scheme, f, err)
    # and the scheme changed the tendencies against the defaults
    d = oracle.OracleModel(c.with_params(vertical_weno=0, momentum_vadv=0))
    d.tendencies()
    field = "GT" if scheme["vertical_weno"] and not scheme["momentum_vadv"] else "Gu"
    assert max_rel(d.get(field), o.get(field)) > 1e-6, scheme


@pytest.mark.parametrize("scheme", VERTICAL_SCHEMES)
@pytest.mark.parametrize("precision", [ocean.OCEAN_FP64, ocean.OCEAN_MIXED])
def test_vertical_schemes_match_oracle(scheme, precision):
    for c, steps in ((_moving_state(inputs.latlon_small_case()).with_params(**scheme), 40),
                     (inputs.box_case().with_params(**scheme), 60)):
        g, o = run_pair(c, precision, steps)
        if precision == ocean.OCEAN_FP64:
            errs = state_errors(g, o)
            assert all(e <= FP64_TOL for e in errs.values()), (c.name, scheme, errs)
        else:
            errs = state_errors(g, o, rel_l2)
            assert all(e <= MIXED_TOL for e in errs.values()), (c.name, scheme, errs)


@pytest.mark.parametrize("shape,periodic", [((37, 23, 5), (False, False)),
                                            ((33, 9, 3), (True, True)),
                                            ((5, 6, 1), (False, False)),
                                            ((64, 4, 2), (True, False))])
@pytest.mark.parametrize("precision", [ocean.OCEAN_FP64, ocean.OCEAN_MIXED])
def test_ragged_and_degenerate_shapes(shape, periodic, precision):
    nx, ny, nz = shape
    rng = np.random.default_rng(nx * 100 + ny)
    T = 10 + 5 * rng.random((nz, ny, nx))
    c = flat_box(nx, ny, nz, periodic_x=periodic[0], periodic_y=periodic[1], T=T,
                 u=0.05 * rng.standard_normal((nz, ny, nx)),
                 v=0.05 * rng.standard_normal((nz, ny, nx)), dt=300.0, n_substeps=10)
    c.depth[:] = 4000.0 * (0.3 + 0.7 * rng.random((ny, nx)))
    c.depth[rng.random((ny, nx)) < 0.15] = 0.0
    g, o = run_pair(c, precision, 10)
    if precision == ocean.OCEAN_FP64:
        errs = state_errors(g, o)
        assert all(e <= FP64_TOL for e in errs.values()), errs
    else:
        errs = state_errors(g, o, rel_l2)
        assert all(e <= MIXED_TOL for e in errs.values()), errs


def test_all_land_domain_is_inert():
    c = flat_box(8, 8, 3)
    c.depth[:] = 0.0
    g = ocean.Ocean(c, precision=ocean.OCEAN_FP64)
    g.step(3)
    for f in ["u", "v", "T", "S", "eta"]:
        assert np.all(g.get(f) == 0.0)


def test_lake_at_rest_gpu_exact():
    for prec in (ocean.OCEAN_FP64, ocean.OCEAN_MIXED):
        c = lake_at_rest()
        g = ocean.Ocean(c, precision=prec)
        T0 = g.get("T")
        g.step(20)
        assert np.all(g.get("u") == 0.0) and np.all(g.get("v") == 0.0)
        assert np.all(g.get("eta") == 0.0)
        assert np.array_equal(g.get("T"), T0)


def test_conservation_gpu():
    c = inputs.latlon_small_case()
    for prec, tol in ((ocean.OCEAN_FP64, 1e-14), (ocean.OCEAN_MIXED, 1e-6)):
        g = ocean.Ocean(c, precision=prec)
        d0 = g.diagnostics()
        g.step(30)
        d1 = g.diagnostics()
        assert not d1["nonfinite"]
        assert abs(d1["tracer_T"] - d0["tracer_T"]) <= tol * abs(d0["tracer_T"])
        assert abs(d1["tracer_S"] - d0["tracer_S"]) <= tol * abs(d0["tracer_S"])


def test_diagnostics_match_oracle():
    c = _moving_state(inputs.latlon_small_case())
    g, o = run_pair(c, ocean.OCEAN_FP64, 5)
    dg, do = g.diagnostics(), o.diagnostics()
    for k in ["tracer_T", "tracer_S", "ke", "max_cfl", "wet_volume"]:
        assert abs(dg[k] - do[k]) <= 1e-10 * abs(do[k]), k
    # sum eta dA is a roundoff-level quantity in a closed basin: compare on the scale of
    # sum |eta| dA
    eta = o.get("eta")
    dlat = (c.y1 - c.y0) / c.ny
    phi = np.radians(c.y0 + (np.arange(c.ny) + 0.5) * dlat)
    area = c.params["radius"] ** 2 * np.cos(phi) * np.radians(360.0 / c.nx) * np.radians(dlat)
    scale = np.sum(np.abs(eta) * area[:, None])
    assert abs(dg["volume_eta"] - do["volume_eta"]) <= 1e-13 * scale


def test_checkpoint_resume_is_bitwise():
    for prec in (ocean.OCEAN_MIXED, ocean.OCEAN_FP64):
        c = _moving_state(inputs.latlon_small_case())
        a = ocean.Ocean(c, precision=prec)
        a.step(20)
        saved = a.checkpoint()
        a.step(20)
        b = ocean.Ocean(c, precision=prec)
        b.restore(saved)
        b.step(20)
        for f in ["u", "v", "T", "S", "eta", "T_anom", "S_anom"]:
            assert np.array_equal(a.get(f), b.get(f)), (prec, f)


def test_health_check_flags_nonfinite_state():
    c = inputs.box_case()
    g = ocean.Ocean(c, precision=ocean.OCEAN_FP64, check_every=1)
    g.step(2)
    # a state whose CFL number exceeds one is reported, not silently advanced
    u = np.full((c.nz, c.ny, c.nx), 200.0)
    g.set("u", u)
    with pytest.raises(ocean.OceanError) as e:
        g.step(1)
    assert e.value.code == -3


@pytest.mark.parametrize("precision,tol", [(ocean.OCEAN_FP64, 1e-13), (ocean.OCEAN_MIXED, 2e-6)])
def test_weno_faces_match_oracle(precision, tol):
    import torch
    rng = np.random.default_rng(5)
    n = 257
    q = np.cumsum(rng.standard_normal(n)) * 0.3
    vel = rng.standard_normal(n)
    inside = (rng.random(n) > 0.1).astype(np.uint8)
    out = ocean.weno_faces(torch.tensor(q), torch.tensor(vel), torch.tensor(inside),
                           precision=precision).cpu().double().numpy()
    ref = np.zeros(n)
    for f in range(n):
        idx = [(f - 3 + m) % n if vel[f] >= 0 else (f + 2 - m) % n for m in range(5)]
        ref[f] = oracle.recon(q[idx], inside[idx])
    assert np.max(np.abs(out - ref)) <= tol * np.max(np.abs(ref))


@pytest.mark.parametrize("precision,tol", [(ocean.OCEAN_FP64, 1e-14), (ocean.OCEAN_MIXED, 1e-6)])
def test_tridiag_batched_matches_dense_solve(precision, tol):
    import torch
    rng = np.random.default_rng(7)
    for n in (1, 2, 5, 48):
        nsys = 333
        a = -rng.uniform(0, 1, (n, nsys))
        c = -rng.uniform(0, 1, (n, nsys))
        b = 1 + np.abs(a) + np.abs(c) + rng.uniform(0, 1, (n, nsys))
        d = rng.standard_normal((n, nsys))
        x = ocean.tridiag_batched(*(torch.tensor(t) for t in (a, b, c, d)),
                                  precision=precision).cpu().double().numpy()
        for s in range(0, nsys, 37):
            A = np.diag(b[:, s]) + np.diag(a[1:, s], -1) + np.diag(c[:-1, s], 1)
            ref = np.linalg.solve(A, d[:, s])
            assert np.max(np.abs(x[:, s] - ref)) <= tol * max(1.0, np.max(np.abs(ref)))


@pytest.mark.slow
def test_latlon_1deg_fp64_10_steps():
    c = _moving_state(inputs.latlon_1deg_case(), amp=0.02)
    g, o = run_pair(c, ocean.OCEAN_FP64, 10)
    errs = state_errors(g, o)
    assert all(e <= FP64_TOL for e in errs.values()), errs


@pytest.mark.gpu
def test_graph_replayed_step_is_bitwise_the_direct_step():
    # on a side stream the step after the Euler start is a CUDA graph per buffer parity;
    # on the legacy default stream (not capturable) every kernel is launched directly
    import torch
    c = _moving_state(inputs.latlon_small_case(seed=21))
    a = ocean.Ocean(c, precision=ocean.OCEAN_MIXED)
    a.step(7)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        b = ocean.Ocean(c, precision=ocean.OCEAN_MIXED)
        b.step(7)
        launches = b.launches
    assert launches == a.launches
    for f in ("u", "v", "T_anom", "S_anom", "eta", "Gu_prev", "GT_prev"):
        assert np.array_equal(a.get(f), b.get(f)), f


@pytest.mark.gpu
def test_wind_stress_replaced_after_creation_matches_the_oracle_built_with_it():
    # the upload path of ocean_set_wind_stress (two device copies and a scatter kernel
    # that scales each column into the padded fields): a model created with one stress
    # and given another before stepping is the oracle built with the second; null arrays
    # mean zero stress
    import ctypes
    import dataclasses
    a = _moving_state(inputs.latlon_small_case())
    rng = np.random.default_rng(11)
    b = dataclasses.replace(a, taux=rng.normal(0.0, 0.1, a.taux.shape),
                            tauy=rng.normal(0.0, 0.1, a.tauy.shape))
    for prec, measure, tol in ((ocean.OCEAN_FP64, max_rel, FP64_TOL),
                               (ocean.OCEAN_MIXED, rel_l2, MIXED_TOL)):
        g = ocean.Ocean(a, precision=prec)
        g.set_wind_stress(b.taux, b.tauy)
        o = oracle.OracleModel(b)
        g.step(10)
        o.step(10)
        errs = state_errors(g, o, measure)
        assert all(e <= tol for e in errs.values()), (prec, errs)
    z = dataclasses.replace(a, taux=np.zeros_like(a.taux), tauy=np.zeros_like(a.tauy))
    g = ocean.Ocean(a, precision=ocean.OCEAN_FP64)
    assert ocean.load().ocean_set_wind_stress(g._h, None, None) == 0
    o = oracle.OracleModel(z)
    g.step(10)
    o.step(10)
    errs = state_errors(g, o)
    assert all(e <= FP64_TOL for e in errs.values()), errs


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [ocean.OCEAN_FP64, ocean.OCEAN_MIXED])
def test_wind_stress_from_float_arrays_is_bitwise_the_double_upload(precision):
    # ocean_set_wind_stress_f32 widens each value to FP64 before scaling it, so float
    # arrays and the double arrays of the same values give the same model, bit for bit
    a = _moving_state(inputs.latlon_small_case())
    rng = np.random.default_rng(5)
    tx = rng.normal(0.0, 0.1, a.taux.shape).astype(np.float32)
    ty = rng.normal(0.0, 0.1, a.tauy.shape).astype(np.float32)
    f = ocean.Ocean(a, precision=precision)
    d = ocean.Ocean(a, precision=precision)
    f.set_wind_stress(tx, ty)                                       # the float32 entry point
    d.set_wind_stress(tx.astype(np.float64), ty.astype(np.float64))
    f.step(5)
    d.step(5)
    for name in ("u", "v", "T_anom", "S_anom", "eta"):
        assert np.array_equal(f.get(name), d.get(name)), name


@pytest.mark.gpu
def test_mixed_diagnostics_agree_with_the_fp64_reduction():
    # the mixed form's reduction (FP32 metrics and column sums, the reference profiles'
    # part of the totals and the wet volume formed once on the host) against the FP64
    # reduction of the same state: the mixed model's fields, widened, set into an FP64
    # model of the same case
    c = _moving_state(inputs.latlon_small_case())
    g = ocean.Ocean(c, precision=ocean.OCEAN_MIXED)
    g.step(3)
    h = ocean.Ocean(c, precision=ocean.OCEAN_FP64)
    for name in ("u", "v", "T", "S", "eta"):
        h.set(name, g.get(name))
    dm, dd = g.diagnostics(), h.diagnostics()
    for k, tol in (("tracer_T", 1e-6), ("tracer_S", 1e-6), ("wet_volume", 1e-12),
                   ("ke", 1e-5), ("max_cfl", 1e-5)):
        assert abs(dm[k] - dd[k]) <= tol * abs(dd[k]), (k, dm[k], dd[k])
    assert not dm["nonfinite"] and not dd["nonfinite"]
