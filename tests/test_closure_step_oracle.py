"""Pins of the oracle's learned-closure step (CPU): a network whose diffusivity is a
constant K2 on top of a Richardson-number closure that gives K1 everywhere is the plain
step with K1 + K2, and a constant tendency correction adds exactly dt * c * (wet volume)
of tracer."""
import math

import numpy as np

import oracle
from oracle import closure as C
from paper_2309_06662_gb300 import inputs

SCALES = dict(kappa=1e-2, gT=1e-6, gS=1e-7, sFT=1, sFS=1, sGT=1, sGS=1)


def _net(nz, hidden, last_bias):
    dims = [6 * nz, hidden, hidden, hidden, 3 * nz]
    params = [(np.zeros((a, b)), np.zeros(b)) for a, b in zip(dims[:-1], dims[1:])]
    params[-1] = (params[-1][0], np.asarray(last_bias, float))
    return params


def _case(K):
    """kappa = K on every interior face: nu0 = nu_b = 0, and a start from rest with
    uniform salinity, so no face turns convective in five steps (convective faces would
    also set nu = kappa_conv, which the network does not touch)."""
    c = inputs.latlon_small_case(seed=12)
    c.S = np.where(c.S != 0.0, 35.0, 0.0)
    return c.with_params(nu0=0.0, nu_b=0.0, kappa_b=K, kappa_conv=K)


def test_learned_diffusivity_adds_to_the_richardson_kappa():
    K1, K2 = 1e-3, 2e-3
    nz = _case(K1).nz
    b = np.zeros(3 * nz)
    b[:nz] = math.log(math.expm1(K2 / SCALES["kappa"]))    # softplus^{-1}(K2 / kappa_scale)
    params = _net(nz, 16, b)
    mu, sigma = np.zeros(6 * nz), np.ones(6 * nz)
    a = oracle.OracleModel(_case(K1 + K2))
    a.step(5)
    m = oracle.OracleModel(_case(K1))
    C.step_learned(m, 5, params, mu, sigma, SCALES, bf16=False)
    for f in ("u", "v", "T", "S", "eta"):
        x, y = m.get(f), a.get(f)
        assert np.max(np.abs(x - y)) <= 1e-13 * max(1.0, np.max(np.abs(y))), f
    # and the diffusivity really matters at this size
    c = oracle.OracleModel(_case(K1))
    c.step(5)
    assert np.max(np.abs(c.get("T") - a.get("T"))) > 1e-9


def test_constant_tendency_correction_adds_dt_c_volume():
    c = inputs.latlon_small_case(seed=13)
    nz = c.nz
    cT = 2e-7
    b = np.zeros(3 * nz)
    b[:nz] = -30.0                                          # negligible learned kappa
    b[nz:2 * nz] = cT / SCALES["gT"]
    params = _net(nz, 16, b)
    m = oracle.OracleModel(c)
    d0 = m.diagnostics()
    C.step_learned(m, 1, params, np.zeros(6 * nz), np.ones(6 * nz), SCALES, bf16=False)
    d1 = m.diagnostics()
    expect = c.params["dt"] * cT * d0["wet_volume"]
    assert abs((d1["tracer_T"] - d0["tracer_T"]) - expect) <= 1e-8 * expect
    assert abs(d1["tracer_S"] - d0["tracer_S"]) <= 1e-14 * d0["tracer_S"]
