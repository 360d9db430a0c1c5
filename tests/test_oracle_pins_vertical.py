"""Pins of the oracle's vertical schemes on stretched levels (no GPU needed).

The adaptive WENO of the paper (Sec. "New numerical methods for finite volume fluid
dynamics on the sphere") is read on stretched levels as: candidate polynomials and ideal
weights from the level thicknesses, smoothness indicators in index space.  The vertical
momentum advection has a centred form and a WENO flux form.  What pins them:
- on uniform levels the coefficients are the textbook Jiang-Shu values;
- on random non-uniform stencils the candidates are exact for quadratics, the
  fifth-order linear combination for quartics, the nonlinear WENO-Z for quadratics and
  its third-order fallback for linear profiles (analytic cell means);
- fifth-order convergence on a smoothly stretched grid, where index-space coefficients
  fall to first order;
- in the model, a tracer linear in z keeps the closed-form vertical flux divergence on
  stretched levels, and stretched coefficients on uniform levels change nothing;
- the momentum term vanishes for a uniform profile, equals w dF/dz for a linear one, and
  both forms converge to w dF/dz.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2309_06662_gb300 import inputs
from tests.oracle_cases import NO_MIXING


def _means(coef, e):
    """Analytic means of the polynomial sum_n coef[n] x^n over the cells of edges e."""
    P = lambda x: sum(c * x ** (n + 1) / (n + 1) for n, c in enumerate(coef))
    return np.array([(P(e[j + 1]) - P(e[j])) / (e[j + 1] - e[j]) for j in range(len(e) - 1)])


def _poly(coef, x):
    return sum(c * x ** n for n, c in enumerate(coef))


def _random_stencil(rng, reverse=False):
    w = rng.uniform(0.4, 2.5, size=5)
    e = np.concatenate([[0.0], np.cumsum(w)])
    if reverse:   # downward stencil: edges decreasing
        e = e[::-1].copy()
    return e, e[3]   # the face downstream of cell 2


def test_uniform_coefficients_are_the_jiang_shu_values():
    e = np.arange(6, dtype=float)
    c, d, c3, d3 = oracle.weno_coeffs(e, 3.0)
    np.testing.assert_allclose(c[0], [1 / 3, -7 / 6, 11 / 6], atol=1e-14)
    np.testing.assert_allclose(c[1], [-1 / 6, 5 / 6, 1 / 3], atol=1e-14)
    np.testing.assert_allclose(c[2], [1 / 3, 5 / 6, -1 / 6], atol=1e-14)
    np.testing.assert_allclose(d, [0.1, 0.6, 0.3], atol=1e-14)
    np.testing.assert_allclose(c3, [[-0.5, 1.5], [0.5, 0.5]], atol=1e-14)
    np.testing.assert_allclose(d3, [1 / 3, 2 / 3], atol=1e-14)
    # and a scaled, shifted, decreasing copy of the same stencil gives the same numbers
    c2, d2, _, _ = oracle.weno_coeffs(100.0 - 7.5 * e, 100.0 - 22.5)
    np.testing.assert_allclose(c2, c, atol=1e-13)
    np.testing.assert_allclose(d2, d, atol=1e-13)


@pytest.mark.parametrize("reverse", [False, True])
def test_stretched_candidates_and_linear_weights_exactness(reverse):
    rng = np.random.default_rng(7 + reverse)
    for _ in range(30):
        e, xf = _random_stencil(rng, reverse)
        c, d, c3, d3 = oracle.weno_coeffs(e, xf)
        for deg in range(5):
            coef = rng.normal(size=deg + 1)
            q = _means(coef, e)
            exact = _poly(coef, xf)
            tol = 1e-11 * (1 + abs(exact) + np.max(np.abs(q)))
            cand = [c[r] @ q[r:r + 3] for r in range(3)]
            if deg <= 2:
                for r in range(3):
                    assert abs(cand[r] - exact) <= tol, (deg, r)
            assert abs(np.dot(d, cand) - exact) <= tol, deg           # fifth order: deg <= 4
            if deg <= 2:
                p3 = [c3[0] @ q[1:3], c3[1] @ q[2:4]]
                assert abs(np.dot(d3, p3) - exact) <= tol, deg        # third order: deg <= 2
            if deg <= 1:
                assert abs(c3[0] @ q[1:3] - exact) <= tol and abs(c3[1] @ q[2:4] - exact) <= tol
        assert abs(d.sum() - 1) < 1e-13 and abs(d3.sum() - 1) < 1e-13


@pytest.mark.parametrize("deg", [0, 1, 2])
def test_stretched_nonlinear_weno_exact_to_degree2(deg):
    rng = np.random.default_rng(30 + deg)
    for _ in range(20):
        e, xf = _random_stencil(rng, reverse=bool(rng.integers(2)))
        coef = rng.normal(size=deg + 1)
        q = _means(coef, e)
        exact = _poly(coef, xf)
        got = oracle.recon_coef(q, [1] * 5, e, xf)
        assert abs(got - exact) <= 1e-11 * (1 + abs(exact)), (deg, got, exact)
        if deg <= 1:   # the third-order scheme's candidates are linear
            got3 = oracle.recon_coef(q, [0, 1, 1, 1, 0], e, xf)
            assert abs(got3 - exact) <= 1e-11 * (1 + abs(exact)), (deg, got3, exact)


def test_uniform_edges_reduce_to_the_index_space_scheme():
    rng = np.random.default_rng(5)
    for _ in range(50):
        q = rng.normal(size=5)
        e = 3.0 + 0.7 * np.arange(6)
        for ins in ([1] * 5, [0, 1, 1, 1, 0], [0, 0, 1, 1, 1]):
            a = oracle.recon_coef(q, ins, e, e[3])
            b = oracle.recon(q, ins)
            assert abs(a - b) <= 1e-13 * (1 + abs(b))


def _stretched_faces(n, s=3.0):
    # the exponential stretching of the configurations' levels, on [0, 1]
    m = np.arange(n + 1) / n
    return (np.exp(s * m) - 1) / (np.exp(s) - 1)


def _max_face_error(n, stretched):
    """Max error of the nonlinear WENO-Z at the interior faces of a stretched grid for the
    cell means of sin(2 pi x), both upwind directions."""
    e = _stretched_faces(n)
    f = lambda x: np.sin(2 * np.pi * x)
    F = lambda x: -np.cos(2 * np.pi * x) / (2 * np.pi)
    q = (F(e[1:]) - F(e[:-1])) / np.diff(e)
    err = 0.0
    for k in range(3, n - 2):    # face e[k] between cells k-1 and k
        up = q[k - 3:k + 2]
        down = q[k - 2:k + 3][::-1]
        if stretched:
            a = oracle.recon_coef(up, [1] * 5, e[k - 3:k + 3], e[k])
            b = oracle.recon_coef(down, [1] * 5, e[k - 2:k + 4][::-1], e[k])
        else:
            a, b = oracle.recon(up, [1] * 5), oracle.recon(down, [1] * 5)
        err = max(err, abs(a - f(e[k])), abs(b - f(e[k])))
    return err


def test_fifth_order_on_stretched_levels():
    ns = [40, 80, 160, 320]
    errs = [_max_face_error(n, True) for n in ns]
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(len(ns) - 1)]
    overall = np.log2(errs[0] / errs[-1]) / (len(ns) - 1)
    assert overall > 4.6 and min(rates) > 4.2, (errs, rates)
    # index-space coefficients on the same grid lose the order
    errs_u = [_max_face_error(n, False) for n in ns]
    rates_u = [np.log2(errs_u[i] / errs_u[i + 1]) for i in range(len(ns) - 1)]
    assert max(rates_u[1:]) < 2.5, (errs_u, rates_u)
    assert errs[-1] < 1e-3 * errs_u[-1]


def test_ideal_weights_positive_on_the_configured_levels():
    for nz, H in ((32, 5000.0), (48, 5000.0), (100, 4000.0)):
        zf = inputs.stretched_z_faces(nz, H)
        for kf in range(3, nz - 2):
            for e in (zf[kf - 3:kf + 3], zf[kf - 2:kf + 4][::-1]):
                _, d, _, d3 = oracle.weno_coeffs(e, zf[kf])
                assert np.all(d > 0) and np.all(d3 > 0), (nz, kf, d, d3)


# ----------------------------------------------------------------------------- in the model

def _column_channel(zf, T_of_z, vertical_weno, nx=16, ny=6):
    """Flat periodic channel (walls in y) on the given levels with u = 0.2 sin(2 pi x / L)
    cos(pi z / H): a divergent flow whose w is non-zero inside the column."""
    nz = len(zf) - 1
    L, H = 4.0e5, -zf[0]
    zc = 0.5 * (zf[1:] + zf[:-1])
    x = (np.arange(nx)) * L / nx              # u-faces
    u = 0.2 * np.sin(2 * np.pi * x / L)[None, None, :] * np.cos(np.pi * zc / H)[:, None, None]
    u = np.broadcast_to(u, (nz, ny, nx)).copy()
    T = np.broadcast_to(T_of_z(zc)[:, None, None], (nz, ny, nx)).copy()
    p = inputs.default_params()
    p.update(NO_MIXING)
    p.update(vertical_weno=vertical_weno, f0=0.0, beta_plane=0.0)
    c = inputs.Case("channel", 0, nx, ny, nz, True, False, 0.0, L, 0.0, L * ny / nx, zf,
                    np.full((ny, nx), H), np.zeros((ny, nx)), np.zeros((ny, nx)), T,
                    np.full((nz, ny, nx), 35.0), p, steps=1)
    c.u = u
    c.v = None
    c.eta = None
    return c


def test_linear_tracer_vertical_flux_closed_form_on_stretched_levels():
    zf = inputs.stretched_z_faces(24, 4000.0)
    b = 2.0e-3
    Tz = lambda z: 5.0 + b * (z + 4000.0)
    for vw in (1, 0):
        o = oracle.OracleModel(_column_channel(zf, Tz, vw))
        o.tendencies()
        G, w = o.get("GT"), o.get("w")
        dz = np.diff(zf)
        zc = 0.5 * (zf[1:] + zf[:-1])
        worst = 0.0
        for k in range(3, 24 - 3):
            wb, wt = w[k], w[k + 1]   # bottom and top faces of level k
            expect = -b * (wt * (zf[k + 1] - zc[k]) - wb * (zf[k] - zc[k])) / dz[k]
            worst = max(worst, np.max(np.abs(G[k] - expect)) / np.max(np.abs(b * w)))
        if vw == 1:
            assert worst < 1e-10, worst
        else:
            assert worst > 1e-3, worst   # index-space weights miss it on stretched levels


def test_stretched_coefficients_change_nothing_on_uniform_levels():
    zf = inputs.uniform_z_faces(16, 4000.0)
    Tz = lambda z: 10.0 + 3.0 * np.sin(z / 700.0)
    G = []
    for vw in (0, 1):
        o = oracle.OracleModel(_column_channel(zf, Tz, vw))
        o.tendencies()
        G.append(o.get("GT"))
    assert np.max(np.abs(G[0] - G[1])) <= 1e-12 * np.max(np.abs(G[0]))


def test_vertical_momentum_advection_uniform_and_linear_profiles():
    rng = np.random.default_rng(3)
    zf = inputs.stretched_z_faces(20, 5000.0)
    zc = 0.5 * (zf[1:] + zf[:-1])
    nz = 20
    for k0 in (0, 4):
        wf = np.concatenate([[0.0], rng.normal(size=nz - 1) * 1e-3, [0.0]])
        wf[:k0 + 1] = 0.0
        va = oracle.vertical_advection_column(zf, np.full(nz, 0.3), k0, wf)
        assert np.max(np.abs(va[k0:])) == 0.0 or np.max(np.abs(va[k0:])) < 1e-18
        # linear profile, constant w on the interior faces: w dF/dz wherever both faces
        # are reconstructed at third order or better
        wc = np.concatenate([[0.0], np.full(nz - 1, 2e-3), [0.0]])
        F = 0.1 + 4e-5 * zc
        for vw, mv in ((1, 1), (1, 0), (0, 0)):
            va = oracle.vertical_advection_column(zf, F, 0, wc, vertical_weno=vw, momentum_vadv=mv)
            for k in range(3, nz - 3):
                assert abs(va[k] - 2e-3 * 4e-5) <= 1e-12 * 8e-8 + 1e-20, (vw, mv, k, va[k])
        va = oracle.vertical_advection_column(zf, F, 0, wc, vertical_weno=0, momentum_vadv=1)
        assert np.max(np.abs(va[3:nz - 3] - 8e-8)) > 1e-10   # index-space flux form is not exact


@pytest.mark.parametrize("mv", [0, 1])
def test_vertical_momentum_advection_converges(mv):
    errs = []
    for nz in (40, 80, 160):
        zf = 1000.0 * (_stretched_faces(nz) - 1.0)
        zc = 0.5 * (zf[1:] + zf[:-1])
        F = np.cos(2 * np.pi * zc / 1000.0)
        wf = 1e-3 * np.sin(np.pi * (zf + 1000.0) / 1000.0)    # zero at both ends
        va = oracle.vertical_advection_column(zf, F, 0, wf, vertical_weno=1, momentum_vadv=mv)
        wcen = 1e-3 * np.sin(np.pi * (zc + 1000.0) / 1000.0)
        exact = wcen * (-2 * np.pi / 1000.0) * np.sin(2 * np.pi * zc / 1000.0)
        inner = slice(nz // 8, nz - nz // 8)
        errs.append(np.max(np.abs(va[inner] - exact[inner])))
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(rates) > 1.8, (errs, rates)


def test_depth_uniform_velocity_has_no_vertical_advection_in_either_form():
    """In the model: with u, v uniform over each column's depth the vertical term is zero
    in both forms, so the two momentum tendencies agree (including the columns' lowest wet
    levels and the surface)."""
    case = inputs.latlon_case(24, 16, 10, 60.0, 4, 1800.0, 10, 50, "vadv", noise=0.05,
                              corr_deg=20.0)
    rng = np.random.default_rng(9)
    u2 = 0.1 * rng.normal(size=(case.ny, case.nx))
    v2 = 0.1 * rng.normal(size=(case.ny, case.nx))
    case.u = np.broadcast_to(u2, (case.nz, case.ny, case.nx)).copy()
    case.v = np.broadcast_to(v2, (case.nz, case.ny, case.nx)).copy()
    G = {}
    for mv in (0, 1):
        o = oracle.OracleModel(case.with_params(momentum_vadv=mv, vertical_weno=1))
        o.tendencies()
        G[mv] = (o.get("Gu"), o.get("Gv"), o.get("w"))
    assert np.max(np.abs(G[0][2])) > 1e-7    # the flow does move vertically
    for a, b in zip(G[0][:2], G[1][:2]):
        assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(a))
