"""Pins of the CPU oracle against what the mathematics fixes (no GPU needed).

Each test checks the oracle against something other than itself: polynomial
exactness and convergence orders of the WENO reconstructions, a dense pivoted
solve for the Thomas algorithm, closed-form solutions of special cases (inertial
oscillation, forward-backward gravity wave, linear pressure gradient), exact
invariants (lake at rest, conservation, free-stream preservation, column integrals
under the implicit solve) and second-order convergence of the full tendencies to
the continuum equations.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from paper_2309_06662_gb300 import inputs
from tests.oracle_cases import NO_MIXING, flat_box, lake_at_rest, seeded_velocity

# ----------------------------------------------------------------------------- WENO


def _cell_avg_poly(c, i):
    a, b = i - 0.5, i + 0.5
    return sum(cn * (b ** (n + 1) - a ** (n + 1)) / (n + 1) for n, cn in enumerate(c))


def _poly(c, x):
    return sum(cn * x ** n for n, cn in enumerate(c))


@pytest.mark.parametrize("deg", [0, 1, 2, 3, 4])
def test_weno5_linear_exact_to_degree4(deg):
    rng = np.random.default_rng(deg)
    for _ in range(20):
        c = rng.normal(size=deg + 1)
        q = [_cell_avg_poly(c, i) for i in range(-2, 3)]
        exact = _poly(c, 0.5)
        got = oracle.weno5(q, linear=True)
        assert abs(got - exact) <= 1e-12 * (1 + abs(exact))


@pytest.mark.parametrize("deg", [0, 1, 2])
def test_weno5_nonlinear_exact_to_degree2(deg):
    rng = np.random.default_rng(10 + deg)
    for _ in range(20):
        c = rng.normal(size=deg + 1)
        q = [_cell_avg_poly(c, i) for i in range(-2, 3)]
        assert abs(oracle.weno5(q) - _poly(c, 0.5)) <= 1e-12 * (1 + abs(_poly(c, 0.5)))


def test_weno5_nonlinear_not_exact_for_cubic():
    # an asymmetric cubic is outside the exactness class of the nonlinear weights
    # (a symmetric one gives beta_0 = beta_2, tau5 = 0 and the linear weights)
    c = [0.1, -0.2, 0.5, 1.0]
    q = [_cell_avg_poly(c, i) for i in range(-2, 3)]
    assert abs(oracle.weno5(q, linear=True) - _poly(c, 0.5)) < 1e-12
    assert abs(oracle.weno5(q) - _poly(c, 0.5)) > 1e-6


@pytest.mark.parametrize("deg,linear", [(0, False), (1, False), (2, True)])
def test_weno3_exactness(deg, linear):
    rng = np.random.default_rng(20 + deg)
    for _ in range(20):
        c = rng.normal(size=deg + 1)
        q = [_cell_avg_poly(c, i) for i in range(-1, 2)]
        assert abs(oracle.weno3(q, linear=linear) - _poly(c, 0.5)) <= 1e-12 * (1 + abs(_poly(c, 0.5)))


def _sine_errors(fn, width, ns):
    errs = []
    for n in ns:
        h = 1.0 / n
        x = (np.arange(n) + 0.5) * h
        avg = (np.cos(2 * np.pi * (x - h / 2)) - np.cos(2 * np.pi * (x + h / 2))) / (2 * np.pi * h)
        e = 0.0
        for i in range(n):
            q = [avg[(i + o) % n] for o in range(-(width // 2), width // 2 + 1)]
            e = max(e, abs(fn(q) - np.sin(2 * np.pi * (i + 1) * h)))
        errs.append(e)
    return np.array(errs)


def test_weno5z_fifth_order_on_smooth_field():
    ns = [20, 40, 80, 160]
    e = _sine_errors(oracle.weno5, 5, ns)
    rates = np.log2(e[:-1] / e[1:])
    assert np.all(np.abs(rates[1:] - 5.0) < 0.3), rates


def test_weno3_linear_third_order():
    e = _sine_errors(lambda q: oracle.weno3(q, linear=True), 3, [20, 40, 80, 160])
    rates = np.log2(e[:-1] / e[1:])
    assert np.all(np.abs(rates[1:] - 3.0) < 0.2), rates


def test_weno_mirror_symmetry():
    # reconstructing the mirrored stencil of -q gives minus the value: no sign bias
    rng = np.random.default_rng(3)
    for _ in range(50):
        q = rng.normal(size=5)
        assert abs(oracle.weno5(q) + oracle.weno5(-q)) < 1e-14
        assert abs(oracle.weno3(q[:3]) + oracle.weno3(-q[:3])) < 1e-14


def test_adaptive_order_selection():
    q = np.array([5.0, -1.0, 2.0, 0.5, 7.0])
    assert oracle.recon(q, [1, 1, 1, 1, 1]) == oracle.weno5(q)
    assert oracle.recon(q, [0, 1, 1, 1, 1]) == oracle.weno3(q[1:4])
    assert oracle.recon(q, [1, 1, 1, 1, 0]) == oracle.weno3(q[1:4])
    assert oracle.recon(q, [1, 1, 1, 0, 1]) == 2.0
    assert oracle.recon(q, [1, 0, 1, 1, 1]) == 2.0


# ----------------------------------------------------------------------------- Thomas


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_thomas_matches_dense_pivoted_solve(n):
    rng = np.random.default_rng(n)
    for _ in range(20):
        a = -rng.uniform(0, 1, n)
        c = -rng.uniform(0, 1, n)
        b = 1.0 + np.abs(a) + np.abs(c) + rng.uniform(0, 1, n)
        d = rng.normal(size=n)
        A = np.diag(b) + np.diag(a[1:], -1) + np.diag(c[:-1], 1)
        x_ref = np.linalg.solve(A, d)
        x = oracle.thomas(a, b, c, d)
        assert np.max(np.abs(x - x_ref)) <= 1e-14 * max(1.0, np.max(np.abs(x_ref)))


# ----------------------------------------------------------------------------- special cases


def test_linear_pressure_gradient_closed_form():
    # T linear in x, uniform in z, S = S0: b = g alpha (T - T0), p = b z, so
    # G_u = -g alpha (T_i - T_{i-1}) z_c / dx exactly (no motion yet).
    nx, ny, nz = 8, 4, 5
    x = np.arange(nx)
    T = 10.0 + 0.3 * x[None, None, :] + np.zeros((nz, ny, nx))
    c = flat_box(nx, ny, nz, T=T, **NO_MIXING)
    m = oracle.OracleModel(c)
    m.tendencies()
    Gu = m.get("Gu")
    p = c.params
    zc = 0.5 * (c.z_faces[1:] + c.z_faces[:-1])
    dx = 1.0e6 / nx
    expect = -p["g"] * p["alpha"] * 0.3 * zc[:, None, None] / dx * np.ones((nz, ny, nx - 1))
    np.testing.assert_allclose(Gu[:, :, 1:], expect, rtol=1e-12, atol=0)
    assert np.all(Gu[:, :, 0] == 0.0)       # wall face
    # and in y, with the sign of the meridional gradient
    T = 10.0 - 0.2 * np.arange(ny)[None, :, None] + np.zeros((nz, ny, nx))
    m = oracle.OracleModel(flat_box(nx, ny, nz, T=T, **NO_MIXING))
    m.tendencies()
    Gv = m.get("Gv")
    dy = 1.0e6 / ny
    expect = p["g"] * p["alpha"] * 0.2 * zc[:, None, None] / dy * np.ones((nz, ny - 1, nx))
    np.testing.assert_allclose(Gv[:, 1:, :], expect, rtol=1e-12, atol=0)


def test_lake_at_rest_stays_at_rest():
    c = lake_at_rest()
    m = oracle.OracleModel(c)
    T0 = m.get("T")
    m.step(20)
    assert np.all(m.get("u") == 0.0)
    assert np.all(m.get("v") == 0.0)
    assert np.all(m.get("eta") == 0.0)
    assert np.array_equal(m.get("T"), T0)


def _inertial_closed_form(w0, fdt, chi, n):
    """AB2 recurrence w^{k+1} = w^k - i f dt [(3/2+chi) w^k - (1/2+chi) w^{k-1}] started by
    one forward-Euler step, solved through its characteristic roots."""
    a, b = 1.5 + chi, 0.5 + chi
    l1, l2 = np.roots([1.0, -(1.0 - 1j * fdt * a), -1j * fdt * b])
    w1 = w0 * (1.0 - 1j * fdt)
    B = (w1 - l1 * w0) / (l2 - l1)
    A = w0 - B
    k = np.arange(n + 1)
    return A * l1 ** k + B * l2 ** k


def test_inertial_oscillation_matches_ab2_roots():
    nx, ny, nz = 4, 4, 3
    dt, f0 = 600.0, 1e-4
    c = flat_box(nx, ny, nz, periodic_x=True, periodic_y=True, u=0.1, v=0.0,
                 dt=dt, f0=f0, beta_plane=0.0)
    m = oracle.OracleModel(c)
    n = 60
    w = _inertial_closed_form(0.1 + 0j, f0 * dt, c.params["chi"], n)
    for k in range(1, n + 1):
        m.step(1)
        u, v = m.get("u"), m.get("v")
        assert np.max(np.abs(u - w[k].real)) < 1e-12
        assert np.max(np.abs(v - w[k].imag)) < 1e-12
    assert np.max(np.abs(m.get("eta"))) < 1e-12


def test_inertial_period_tends_to_2pi_over_f():
    f0 = 1e-4
    phases = []
    for dt in (400.0, 200.0):
        c = flat_box(2, 2, 2, periodic_x=True, periodic_y=True, u=0.1, v=0.0, dt=dt, f0=f0,
                     beta_plane=0.0)
        m = oracle.OracleModel(c)
        nsteps = int(round(2000 * 200 / dt))
        m.step(nsteps)
        ang = math.atan2(m.get("v")[0, 0, 0], m.get("u")[0, 0, 0])
        expect = -f0 * nsteps * dt
        err = (ang - expect + math.pi) % (2 * math.pi) - math.pi
        phases.append(abs(err))
    # the phase error after a fixed time shrinks at second order in dt
    assert phases[1] < phases[0] / 3.0
    assert phases[1] < 0.05


def test_gravity_wave_forward_backward_closed_form():
    # flat bottom, f = 0, one Fourier mode of eta in a periodic channel: the sub-cycle's
    # averaged output equals the mean of A^m over m = 1..N_s, with A the forward-backward
    # amplification matrix whose eigenvalues satisfy cos(w dtau) = 1 - (dtau w_s)^2 / 2,
    # w_s = 2 sqrt(gH) sin(k dx / 2) / dx.
    nx, ny, nz, H = 64, 3, 2, 4000.0
    L = 6.4e6
    ns, dt = 30, 900.0
    c = flat_box(nx, ny, nz, L=L, H=H, periodic_x=True, dt=dt, n_substeps=ns)
    m = oracle.OracleModel(c)
    dx = L / nx
    g = c.params["g"]
    dtau = 2 * dt / (ns + 1)
    for mode in (1, 5, 17):
        kx = 2 * math.pi * mode / L
        x = (np.arange(nx) + 0.5) * dx
        eta0 = 0.01 * np.cos(kx * x)[None, :] * np.ones((ny, 1))
        zeros = np.zeros((ny, nx))
        e, Ub, Vb = m.barotropic(eta0, zeros, zeros, zeros, zeros)
        s = 2 * math.sin(kx * dx / 2) / dx
        A = np.array([[1.0, -1j * dtau * s], [-1j * dtau * g * H * s, 1.0 - dtau ** 2 * g * H * s ** 2]])
        lam, V = np.linalg.eig(A)
        ws = math.sqrt(g * H) * s
        assert np.allclose(np.cos(np.angle(lam)), 1 - 0.5 * (dtau * ws) ** 2)
        assert np.allclose(np.abs(lam), 1.0)
        geo = np.array([np.sum(l ** np.arange(1, ns + 1)) / ns for l in lam])
        Mbar = V @ np.diag(geo) @ np.linalg.inv(V)
        hat = Mbar @ np.array([0.01, 0.0])
        expect_eta = np.real(hat[0] * np.exp(1j * kx * x))
        expect_U = np.real(hat[1] * np.exp(1j * kx * (x - dx / 2)))
        np.testing.assert_allclose(e[1], expect_eta, atol=1e-13)
        np.testing.assert_allclose(Ub[1], expect_U, atol=1e-12 * g * H * 0.01 / math.sqrt(g * H))
        assert np.all(Vb == 0.0)
    # the continuum phase speed sqrt(gH) is reached at second order in k dx
    kdx = np.array([0.2, 0.1])
    c_disc = np.sqrt(g * H) * np.sin(kdx / 2) / (kdx / 2)
    err = np.abs(c_disc / math.sqrt(g * H) - 1)
    assert 3.9 < err[0] / err[1] < 4.1


# ----------------------------------------------------------------------------- invariants


def test_conservation_closed_basin():
    c = inputs.latlon_small_case()
    m = oracle.OracleModel(c)
    d0 = m.diagnostics()
    m.step(30)
    d1 = m.diagnostics()
    assert not d1["nonfinite"]
    assert abs(d1["tracer_T"] - d0["tracer_T"]) <= 1e-14 * abs(d0["tracer_T"])
    assert abs(d1["tracer_S"] - d0["tracer_S"]) <= 1e-14 * abs(d0["tracer_S"])
    eta = m.get("eta")
    assert np.max(np.abs(eta)) > 1e-4            # the free surface did move
    dy = c.params["radius"] * math.radians((c.y1 - c.y0) / c.ny)
    phi = np.radians(c.y0 + (np.arange(c.ny) + 0.5) * (c.y1 - c.y0) / c.ny)
    area = c.params["radius"] * np.cos(phi) * math.radians(360.0 / c.nx) * dy
    scale = np.sum(np.abs(eta) * area[:, None])
    assert abs(d1["volume_eta"]) <= 1e-13 * scale
    assert d1["ke"] > 0


def test_free_stream_preservation_below_the_surface():
    # a uniform tracer in any (masked) velocity field: with w from continuity, every
    # cell below the top level has zero advective tendency
    c = inputs.latlon_small_case(seed=9)
    c.T[:] = 12.5
    c.S[:] = 35.0
    c.u, c.v = seeded_velocity(c, 5)
    m = oracle.OracleModel(c)
    m.tendencies()
    G = m.get("GT")
    assert np.max(np.abs(G[:-1])) < 1e-12 * 12.5 * 0.1 / 1e4
    assert np.max(np.abs(G[-1])) > 0         # the surface layer sees w at the top face


def test_implicit_solve_column_integral_and_dense_solve():
    # with u = v = 0 the first step changes T only through the backward-Euler solve
    c = inputs.latlon_small_case(seed=4)
    m = oracle.OracleModel(c)
    m.tendencies()
    kap = m.get("kappa")
    T0 = m.get("T")
    m.step(1)
    T1 = m.get("T")
    zf = c.z_faces
    dz = np.diff(zf)
    zc = 0.5 * (zf[1:] + zf[:-1])
    dt = c.params["dt"]
    checked = 0
    for (j, i) in [(5, 5), (10, 30), (20, 60), (30, 11)]:
        kb = m.kbot(i, j)
        if kb >= c.nz:
            continue
        col0, col1 = T0[kb:, j, i], T1[kb:, j, i]
        assert abs(np.sum(dz[kb:] * col1) - np.sum(dz[kb:] * col0)) <= 1e-14 * np.sum(dz[kb:] * np.abs(col0))
        n = c.nz - kb
        A = np.eye(n)
        for r in range(n):
            k = kb + r
            if r > 0:
                lo = dt * kap[k, j, i] / (dz[k] * (zc[k] - zc[k - 1]))
                A[r, r] += lo
                A[r, r - 1] -= lo
            if k < c.nz - 1:
                hi = dt * kap[k + 1, j, i] / (dz[k] * (zc[k + 1] - zc[k]))
                A[r, r] += hi
                A[r, r + 1] -= hi
        np.testing.assert_allclose(col1, np.linalg.solve(A, col0), rtol=1e-13)
        checked += 1
    assert checked >= 3


def test_richardson_closure_special_cases():
    p = inputs.default_params()
    nx, ny, nz = 3, 3, 4
    # (a) unstable stratification -> convective value
    T = 10.0 - 0.5 * np.arange(nz)[:, None, None] + np.zeros((nz, ny, nx))
    m = oracle.OracleModel(flat_box(nx, ny, nz, T=T))
    m.tendencies()
    assert np.all(m.get("kappa")[1:] == p["kappa_conv"])
    assert np.all(m.get("nu")[1:] == p["kappa_conv"])
    assert np.all(m.get("kappa")[0] == 0.0)       # sea-floor face carries no mixing
    # (b) neutral stratification (N^2 = 0): Ri = 0
    m = oracle.OracleModel(flat_box(nx, ny, nz))
    m.tendencies()
    np.testing.assert_allclose(m.get("nu")[1:], p["nu0"] + p["nu_b"], rtol=1e-15)
    np.testing.assert_allclose(m.get("kappa")[1:], p["nu0"] + p["nu_b"] + p["kappa_b"], rtol=1e-15)
    # (c) Ri = 1 exactly: N^2 = S^2 with a uniform shear in u
    H = 4000.0
    dzf = H / nz
    dT = 0.5
    n2 = p["g"] * p["alpha"] * dT / dzf
    du = math.sqrt(n2) * dzf
    T = 10.0 + dT * np.arange(nz)[:, None, None] + np.zeros((nz, ny, nx))
    u = du * np.arange(nz)[:, None, None] + np.zeros((nz, ny, nx))
    m = oracle.OracleModel(flat_box(nx, ny, nz, H=H, T=T, u=u, periodic_x=True))
    m.tendencies()
    q = 1 + p["ri_a"]
    nu = p["nu0"] / q ** 2 + p["nu_b"]
    np.testing.assert_allclose(m.get("nu")[1:], nu, rtol=1e-12)
    np.testing.assert_allclose(m.get("kappa")[1:], nu / q + p["kappa_b"], rtol=1e-12)


# ----------------------------------------------------------------------------- convergence


def _analytic_fields():
    sp = pytest.importorskip("sympy")
    x, y, z = sp.symbols("x y z", real=True)
    L, H = 1.0e6, 2000.0
    k, l = 2 * sp.pi / L, 2 * sp.pi / L
    U0, V0 = 0.2, 0.15
    u = U0 * sp.cos(k * x) * sp.cos(l * y) * (0.3 + sp.cos(sp.pi * z / H))
    v = V0 * sp.sin(k * x) * sp.sin(l * y) * (0.5 + sp.cos(2 * sp.pi * z / H))
    div = sp.diff(u, x) + sp.diff(v, y)
    zz = sp.symbols("zz", real=True)
    w = -sp.integrate(div.subs(z, zz), (zz, -H, z))
    T = 10.0 + 2.0 * sp.sin(k * x + 0.3) * sp.cos(l * y) * sp.cos(sp.pi * z / (2 * H)) + 3.0 * z / H
    p = dict(g=9.80665, alpha=2e-4, f0=1e-4)
    b = p["g"] * p["alpha"] * (T - 10.0)
    pres = -sp.integrate(b.subs(z, zz), (zz, z, 0))
    f = p["f0"]
    Gu = -(u * sp.diff(u, x) + v * sp.diff(u, y) + w * sp.diff(u, z)) + f * v - sp.diff(pres, x)
    Gv = -(u * sp.diff(v, x) + v * sp.diff(v, y) + w * sp.diff(v, z)) - f * u - sp.diff(pres, y)
    GT = -(u * sp.diff(T, x) + v * sp.diff(T, y) + w * sp.diff(T, z))
    fn = lambda e: sp.lambdify((x, y, z), e, "numpy")
    return dict(L=L, H=H, u=fn(u), v=fn(v), T=fn(T), Gu=fn(Gu), Gv=fn(Gv), GT=fn(GT))


def _discrete_error(F, n):
    nz = n // 2
    L, H = F["L"], F["H"]
    dx = L / n
    dz = H / nz
    xc = (np.arange(n) + 0.5) * dx
    xf = np.arange(n) * dx
    zc = -H + (np.arange(nz) + 0.5) * dz
    Z, Y, X = np.meshgrid(zc, xc, xc, indexing="ij")
    _, Yf, Xf = np.meshgrid(zc, xf, xf, indexing="ij")
    u = F["u"](Xf, Y, Z)
    v = F["v"](X, Yf, Z)
    T = F["T"](X, Y, Z)
    c = flat_box(n, n, nz, L=L, H=H, periodic_x=True, periodic_y=True, T=T, u=u, v=v,
                 f0=1e-4, beta_plane=0.0)
    m = oracle.OracleModel(c)
    m.tendencies()
    # levels within three cells of the sea floor or the surface use the reduced-order
    # vertical reconstructions (first order at the edge), whose O(h) face errors give an
    # O(1) flux-divergence error there by design; the interior uses full WENO5
    inner = slice(3, nz - 3)
    scale_u = np.max(np.abs(F["Gu"](Xf, Y, Z)))
    eu = np.max(np.abs(m.get("Gu") - F["Gu"](Xf, Y, Z))[inner]) / scale_u
    ev = np.max(np.abs(m.get("Gv") - F["Gv"](X, Yf, Z))[inner]) / np.max(np.abs(F["Gv"](X, Yf, Z)))
    eT = np.max(np.abs(m.get("GT") - F["GT"](X, Y, Z))[inner]) / np.max(np.abs(F["GT"](X, Y, Z)))
    return np.array([eu, ev, eT])


@pytest.mark.slow
def test_tendencies_converge_to_continuum_at_second_order():
    F = _analytic_fields()
    e1 = _discrete_error(F, 48)
    e2 = _discrete_error(F, 96)
    ratio = e1 / e2
    assert np.all(e2 < 2e-3), e2
    assert np.all(ratio > 2.8), (e1, e2, ratio)      # second order: 4 asymptotically
