"""Pins of the oracle's forcing, spherical metrics, Coriolis terms, diagnostics and
averaging filter against closed forms (CPU only).

Every expected value below is written from the continuous or discrete definition of
the term it checks (product-form metrics R cos(phi) dlambda, R dphi; Coriolis
2 Omega sin(phi) at the latitude of each staggered point; wind stress entering the top
layer as tau / (rho0 dz_top)), evaluated on states chosen so that every other term of
the step vanishes.  A wrong latitude (row centre against face), a wrong layer thickness,
a dropped factor of the metric, a sign error or a wrong averaging moment fails at least
one of them.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from paper_2309_06662_gb300 import inputs
from tests.oracle_cases import NO_MIXING, flat_box, flat_latlon

R_E = inputs.default_params()["radius"]
OMEGA = inputs.default_params()["omega"]


def _lat(c):
    """Row-centre and south-face latitudes (radians) and spacings of a lat-lon case."""
    dphi = math.radians((c.y1 - c.y0) / c.ny)
    phic = np.radians(c.y0 + (np.arange(c.ny) + 0.5) * (c.y1 - c.y0) / c.ny)
    phif = np.radians(c.y0 + np.arange(c.ny + 1) * (c.y1 - c.y0) / c.ny)
    dlam = math.radians((c.x1 - c.x0) / c.nx)
    return phic, phif, dphi, dlam


# ----------------------------------------------------------------------------- wind stress


@pytest.mark.parametrize("filt", [0, 1])
@pytest.mark.parametrize("axis", ["x", "y"])
def test_wind_stress_accelerates_the_top_layer_only(axis, filt):
    # doubly periodic box, f = 0, uniform T and S, no mixing, stretched levels (so the top
    # layer is thinner than any other): a uniform stress tau drives only the top level,
    # du/dt = tau / (rho0 dz_top); the barotropic mode takes U^{n+1} = U^n + dt tau / rho0
    # (the average's first moment is dt), so the correction is zero and after n steps
    # u_top = n dt tau / (rho0 dz_top) exactly, every other level at rest
    nx, ny, nz = 6, 5, 7
    zf = inputs.stretched_z_faces(nz, 4000.0, 3.0)
    dz = np.diff(zf)
    tau = 0.08
    tx = np.full((ny, nx), tau if axis == "x" else 0.0)
    ty = np.full((ny, nx), tau if axis == "y" else 0.0)
    c = flat_box(nx, ny, nz, periodic_x=True, periodic_y=True, taux=tx, tauy=ty, f0=0.0,
                 beta_plane=0.0, dt=600.0, n_substeps=12, baro_filter=filt, **NO_MIXING)
    c.z_faces = zf
    m = oracle.OracleModel(c)
    p = c.params
    m.tendencies()
    G = m.get("Gu" if axis == "x" else "Gv")
    expect_top = tau / (p["rho0"] * dz[-1])
    np.testing.assert_allclose(G[-1], expect_top, rtol=1e-14)
    assert np.all(G[:-1] == 0.0)
    assert np.all(m.get("Gv" if axis == "x" else "Gu") == 0.0)
    for n in (1, 2, 3):
        m.step(1)
        vel = m.get("u" if axis == "x" else "v")
        np.testing.assert_allclose(vel[-1], n * p["dt"] * expect_top, rtol=1e-12)
        assert np.max(np.abs(vel[:-1])) <= 1e-12 * n * p["dt"] * expect_top
        assert np.max(np.abs(m.get("v" if axis == "x" else "u"))) == 0.0
        assert np.max(np.abs(m.get("eta"))) <= 1e-15


# ----------------------------------------------------------------------------- metrics


def test_cell_areas_sum_to_the_closed_form_band_area():
    # sum over a full band of the product-form areas R^2 cos(phi_c) dlambda dphi: the
    # midpoint sum of cos has the closed form (sin phi1 - sin phi0) (dphi/2)/sin(dphi/2),
    # and tends to the spherical band area 2 pi R^2 (sin phi1 - sin phi0) at second order
    H = 3000.0
    errs = []
    for ny in (20, 40):
        c = flat_latlon(16, ny, 2, lat0=-50.0, lat1=70.0, H=H)
        m = oracle.OracleModel(c)
        vol = m.diagnostics()["wet_volume"]
        s1, s0 = math.sin(math.radians(70.0)), math.sin(math.radians(-50.0))
        dphi = math.radians(120.0 / ny)
        closed = H * R_E ** 2 * 2 * math.pi * (s1 - s0) * (dphi / 2) / math.sin(dphi / 2)
        assert abs(vol - closed) <= 1e-13 * closed
        errs.append(abs(vol / (H * 2 * math.pi * R_E ** 2 * (s1 - s0)) - 1.0))
    assert 3.9 < errs[0] / errs[1] < 4.1


def test_zonally_uniform_zonal_flow_has_no_divergence():
    # u = u(j, k) uniform along each row: every cell's zonal transports cancel, so w = 0
    rng = np.random.default_rng(2)
    c = flat_latlon(12, 10, 4, u=0.3 * rng.standard_normal((4, 10, 1)))
    m = oracle.OracleModel(c)
    m.tendencies()
    assert np.all(m.get("w") == 0.0)


def test_coriolis_at_u_rows_from_meridional_flow():
    # u = 0 and a meridional flow v(j), uniform in x and z: zero vorticity, no zonal
    # gradient of kinetic energy or pressure, no vertical advection of u, so
    # G_u = f(phi_c) * (v_j + v_{j+1}) / 2 with f at the row-centre latitude
    nx, ny, nz = 8, 12, 3
    rng = np.random.default_rng(4)
    vj = 0.2 * rng.standard_normal(ny)
    vj[0] = 0.0                                     # the south wall face
    c = flat_latlon(nx, ny, nz, v=vj[None, :, None], **NO_MIXING)
    m = oracle.OracleModel(c)
    m.tendencies()
    phic, _, _, _ = _lat(c)
    vn = np.append(vj[1:], 0.0)                     # the north face of each row
    expect = 2 * OMEGA * np.sin(phic) * 0.5 * (vj + vn)
    Gu = m.get("Gu")
    np.testing.assert_allclose(Gu, np.broadcast_to(expect[None, :, None], Gu.shape),
                               rtol=1e-13, atol=1e-13 * np.max(np.abs(expect)))


def test_solid_body_zonal_flow_vorticity_and_coriolis_at_v_faces():
    # u = U0 cos(phi_c), v = 0, uniform in x and z: w = 0 and
    #   G_v(j) = -(zeta_j + f(phi_f)) (u_{j-1} + u_j)/2 - (K_j - K_{j-1})/dy,
    #   zeta_j = -(dx_c(j) u_j - dx_c(j-1) u_{j-1}) / (dx_v(j) dy),  K_j = u_j^2 / 2,
    # with dx_c = R cos(phi_c) dlambda, dx_v = R cos(phi_f) dlambda, dy = R dphi and f at
    # the face latitude; the discrete zeta tends to the continuum 2 U0 sin(phi)/R
    nx, ny, nz = 8, 18, 2
    U0 = 0.4
    c0 = flat_latlon(nx, ny, nz, lat0=-70.0, lat1=65.0)
    phic, phif, dphi, dlam = _lat(c0)
    uj = U0 * np.cos(phic)
    c = flat_latlon(nx, ny, nz, lat0=-70.0, lat1=65.0, u=uj[None, :, None], **NO_MIXING)
    m = oracle.OracleModel(c)
    m.tendencies()
    assert np.all(m.get("w") == 0.0)
    assert np.max(np.abs(m.get("Gu"))) <= 1e-18
    dy = R_E * dphi
    dxc = R_E * np.cos(phic) * dlam
    dxv = R_E * np.cos(phif) * dlam
    j = np.arange(1, ny)
    zeta = -(dxc[j] * uj[j] - dxc[j - 1] * uj[j - 1]) / (dxv[j] * dy)
    K = 0.5 * uj ** 2
    expect = -(zeta + 2 * OMEGA * np.sin(phif[j])) * 0.5 * (uj[j - 1] + uj[j]) - (K[j] - K[j - 1]) / dy
    Gv = m.get("Gv")
    np.testing.assert_allclose(Gv[:, 1:, :], np.broadcast_to(expect[None, :, None], (nz, ny - 1, nx)),
                               rtol=1e-12)
    assert np.all(Gv[:, 0, :] == 0.0)
    # second-order agreement of the corner vorticity with the continuum
    cont = 2 * U0 * np.sin(phif[j]) / R_E
    assert np.max(np.abs(zeta - cont)) < 0.01 * np.max(np.abs(cont))


def test_barotropic_continuity_and_gradient_use_the_spherical_metrics():
    # one substep (N_s = 1, dtau = dt) from a uniform meridional transport V0:
    #   eta(j) = -dt / A_c(j) [dx_v(j+1) V_{j+1} - dx_v(j) V_j]   (walls carry V = 0)
    # and from a zonal wave eta0 cos(lambda) at rest:
    #   U(i, j) = -dt g H (eta_i - eta_{i-1}) / dx_c(j),  V(i, j) = 0
    nx, ny, H = 10, 9, 2500.0
    dt = 300.0
    c = flat_latlon(nx, ny, 2, lat0=-40.0, lat1=50.0, H=H, dt=dt, n_substeps=1)
    phic, phif, dphi, dlam = _lat(c)
    m = oracle.OracleModel(c)
    g = c.params["g"]
    V0 = 3.0
    V = np.full((ny, nx), V0)
    V[0, :] = 0.0
    z = np.zeros((ny, nx))
    e, Ub, Vb = m.barotropic(z, z, V, z, z)
    dxv = R_E * np.cos(phif) * dlam
    Ac = R_E * np.cos(phic) * dlam * R_E * dphi
    Vn = np.append(np.full(ny - 1, V0), 0.0)
    Vs = np.concatenate([[0.0], np.full(ny - 1, V0)])
    expect = -dt / Ac * (dxv[1:] * Vn - dxv[:-1] * Vs)
    np.testing.assert_allclose(e, np.broadcast_to(expect[:, None], e.shape), rtol=1e-12)
    lam = np.radians((np.arange(nx) + 0.5) * 360.0 / nx)
    eta0 = 0.02 * np.cos(lam)[None, :] + np.zeros((ny, 1))
    e, Ub, Vb = m.barotropic(eta0, z, z, z, z)
    dxc = R_E * np.cos(phic) * dlam
    expect_U = -dt * g * H * (eta0 - np.roll(eta0, 1, axis=1)) / dxc[:, None]
    np.testing.assert_allclose(Ub, expect_U, rtol=1e-12, atol=1e-15)
    assert np.all(Vb == 0.0)
    np.testing.assert_allclose(e, eta0, rtol=0, atol=1e-17)


def test_tracer_surface_dilution_uses_face_widths():
    # uniform tracer T0 in a uniform meridional flow v0 on the sphere (flat bottom, rigid
    # advective lid): every level below the top is free-stream preserved, and the top cell
    # takes the whole column's horizontal convergence,
    #   G_T(top, j) = -T0 v0 H (dx_v(j+1)[j+1 < ny] - dx_v(j)[j > 0]) / (A_c(j) dz_top)
    nx, ny, nz, H = 6, 8, 4, 3000.0
    T0, v0 = 7.5, 0.15
    vj = np.full(ny, v0)
    vj[0] = 0.0
    c = flat_latlon(nx, ny, nz, lat0=-30.0, lat1=60.0, H=H, T=T0, v=vj[None, :, None], **NO_MIXING)
    m = oracle.OracleModel(c)
    m.tendencies()
    phic, phif, dphi, dlam = _lat(c)
    dxv = R_E * np.cos(phif) * dlam
    Ac = R_E * np.cos(phic) * dlam * R_E * dphi
    north = np.append(dxv[1:ny], 0.0) * np.append(vj[1:], 0.0)
    south = dxv[:ny] * vj
    expect = -T0 * H * (north - south) / (Ac * (H / nz))
    G = m.get("GT")
    np.testing.assert_allclose(G[-1], np.broadcast_to(expect[:, None], (ny, nx)), rtol=1e-11)
    assert np.max(np.abs(G[:-1])) <= 1e-12 * np.max(np.abs(expect))


# ----------------------------------------------------------------------------- diagnostics


def test_kinetic_energy_and_cfl_on_the_sphere_closed_form():
    # u = u0 on every u-face (periodic), v = v0 on every interior v-face:
    #   KE = u0^2/2 H dy sum_j nx dx_c(j) + v0^2/2 H dy sum_{j=1}^{ny-1} nx dx_v(j)
    # and, with v = 0, the largest CFL number is u0 dt / min_j dx_c(j)
    nx, ny, nz, H = 12, 10, 3, 2000.0
    u0, v0 = 0.25, -0.1
    c = flat_latlon(nx, ny, nz, lat0=-60.0, lat1=75.0, H=H, u=u0, v=v0)
    m = oracle.OracleModel(c)
    phic, phif, dphi, dlam = _lat(c)
    dy = R_E * dphi
    dxc = R_E * np.cos(phic) * dlam
    dxv = R_E * np.cos(phif) * dlam
    ke = 0.5 * u0 ** 2 * H * dy * nx * dxc.sum() + 0.5 * v0 ** 2 * H * dy * nx * dxv[1:ny].sum()
    d = m.diagnostics()
    assert abs(d["ke"] - ke) <= 1e-13 * ke
    c2 = flat_latlon(nx, ny, nz, lat0=-60.0, lat1=75.0, H=H, u=u0)
    d2 = oracle.OracleModel(c2).diagnostics()
    assert abs(d2["max_cfl"] - u0 * c.params["dt"] / dxc.min()) <= 1e-14 * d2["max_cfl"]
    assert abs(d2["ke"] - 0.5 * u0 ** 2 * H * dy * nx * dxc.sum()) <= 1e-13 * d2["ke"]


def test_vertical_cfl_in_a_closed_box_closed_form():
    # a walled box on stretched levels with v = v0 on the interior v-faces: the first and
    # last rows see a horizontal divergence of +-v0 dz_k/dy in level k, so w on the bottom
    # face of level k there is -+v0/dy times the thickness of the levels below, and the
    # largest CFL number is v0 dt/dy max(1, max_k (z_k^bottom + H)/dz_k)
    nx, ny, nz, L, H = 5, 6, 5, 6.0e5, 2000.0
    v0 = 0.05
    c = flat_box(nx, ny, nz, L=L, H=H, v=v0)
    c.z_faces = inputs.stretched_z_faces(nz, H, 3.0)
    dz = np.diff(c.z_faces)
    d = oracle.OracleModel(c).diagnostics()
    dy = L / ny
    ratio = max(1.0, max((c.z_faces[k] + H) / dz[k] for k in range(nz)))
    assert abs(d["max_cfl"] - ratio * v0 * c.params["dt"] / dy) <= 1e-13 * d["max_cfl"]
    ke = 0.5 * v0 ** 2 * (ny - 1) * nx * (L / nx) * dy * H
    assert abs(d["ke"] - ke) <= 1e-13 * ke


# ----------------------------------------------------------------------------- averaging filter


@pytest.mark.parametrize("ns", [1, 2, 6, 30, 60])
def test_equal_weights_are_the_boxcar(ns):
    a, mom = oracle.filter_weights(ns, 0)
    np.testing.assert_allclose(a, 1.0 / ns, rtol=1e-15)
    assert abs(mom - (ns + 1) / 2.0) <= 1e-13 * ns


@pytest.mark.parametrize("ns", [6, 20, 30, 60])
def test_power_law_weights(ns):
    # Shchepetkin & McWilliams (2005) shape x^2 (1 - x^4) - 0.284 x over its support
    # (0, x*), x* the root of x - x^5 = 0.284 above 5^(-1/4), sampled at m x*/(ns+1)
    a, mom = oracle.filter_weights(ns, 1)
    assert abs(a.sum() - 1.0) <= 1e-14
    assert abs(mom - np.sum(np.arange(1, ns + 1) * a)) <= 1e-12 * mom
    roots = np.roots([-1.0, 0, 0, 0, 1.0, -0.284])
    xs = max(r.real for r in roots if abs(r.imag) < 1e-12 and 5 ** -0.25 < r.real < 1)
    x = np.arange(1, ns + 1) * xs / (ns + 1)
    s = x ** 2 * (1 - x ** 4) - 0.284 * x
    np.testing.assert_allclose(a, s / s.sum(), rtol=1e-10, atol=1e-14)
    # negative lobe first, one positive main lobe; the centroid sits past the middle
    sign_changes = np.count_nonzero(np.diff(np.sign(a)) != 0)
    assert a[0] < 0 and sign_changes == 1
    assert (ns + 1) / 2 < mom < ns


def test_power_law_filter_second_order_for_slow_modes_and_damps_fast_ones():
    # sum a = 1 and sum a m dtau = dt make the filtered response of a slow oscillation
    # e^{i w t} equal to e^{i w dt} up to O((w dt)^2); a mode near the substep's limit
    # is damped far more than by the boxcar
    ns, dt = 30, 1.0
    a1, mom1 = oracle.filter_weights(ns, 1)
    a0, mom0 = oracle.filter_weights(ns, 0)
    m = np.arange(1, ns + 1)
    errs = []
    for w in (0.02, 0.01):
        resp = np.sum(a1 * np.exp(1j * w * m * dt / mom1))
        errs.append(abs(resp - np.exp(1j * w * dt)))
    assert 3.8 < errs[0] / errs[1] < 4.2
    fast0 = abs(np.sum(a0 * np.exp(1j * 2.0 * m)))
    fast1 = abs(np.sum(a1 * np.exp(1j * 2.0 * m)))
    assert fast1 < 0.5 * fast0


def test_gravity_wave_closed_form_with_power_law_average():
    # the sub-cycle's averaged output is sum_m a_m A^m applied to the initial mode, with A
    # the forward-backward amplification matrix and dtau = dt / sum_m m a_m
    nx, ny, nz, H = 64, 3, 2, 4000.0
    L = 6.4e6
    ns, dt = 30, 900.0
    c = flat_box(nx, ny, nz, L=L, H=H, periodic_x=True, dt=dt, n_substeps=ns, baro_filter=1)
    m = oracle.OracleModel(c)
    a, mom = oracle.filter_weights(ns, 1)
    dtau = dt / mom
    dx = L / nx
    g = c.params["g"]
    for mode in (1, 7, 19):
        kx = 2 * math.pi * mode / L
        x = (np.arange(nx) + 0.5) * dx
        eta0 = 0.01 * np.cos(kx * x)[None, :] * np.ones((ny, 1))
        zeros = np.zeros((ny, nx))
        e, Ub, Vb = m.barotropic(eta0, zeros, zeros, zeros, zeros)
        s = 2 * math.sin(kx * dx / 2) / dx
        A = np.array([[1.0, -1j * dtau * s], [-1j * dtau * g * H * s, 1.0 - dtau ** 2 * g * H * s ** 2]])
        Mbar = sum(a[q] * np.linalg.matrix_power(A, q + 1) for q in range(ns))
        hat = Mbar @ np.array([0.01, 0.0])
        np.testing.assert_allclose(e[1], np.real(hat[0] * np.exp(1j * kx * x)), atol=1e-13)
        np.testing.assert_allclose(Ub[1], np.real(hat[1] * np.exp(1j * kx * (x - dx / 2))),
                                   atol=1e-12 * math.sqrt(g * H) * 0.01)


def test_inertial_oscillation_with_power_law_average():
    # uniform flow on an f-plane: the barotropic correction vanishes whenever the average's
    # first moment is dt, so the AB2 closed form holds with the power-law filter too
    from tests.test_oracle_pins import _inertial_closed_form
    dt, f0 = 600.0, 1e-4
    c = flat_box(4, 4, 3, periodic_x=True, periodic_y=True, u=0.1, v=0.0, dt=dt, f0=f0,
                 beta_plane=0.0, baro_filter=1)
    m = oracle.OracleModel(c)
    n = 30
    w = _inertial_closed_form(0.1 + 0j, f0 * dt, c.params["chi"], n)
    for k in range(1, n + 1):
        m.step(1)
        assert np.max(np.abs(m.get("u") - w[k].real)) < 1e-12
        assert np.max(np.abs(m.get("v") - w[k].imag)) < 1e-12


# ----------------------------------------------------------------------------- masks and flags


def test_full_cell_bathymetry_masks():
    # a cell is wet when its centre lies above the sea floor, and columns shallower than
    # min_depth are land: with faces at -4000, -3000, ..., 0 (centres -3500 .. -500), a
    # depth of 2600 m wets the three top cells (kb = 1), 500 m wets none (the centre sits
    # exactly on the floor), 40 m is land
    nx, ny, nz = 5, 1, 4
    c = flat_box(nx, ny, nz, H=4000.0)
    c.depth[0, :] = [4000.0, 2600.0, 501.0, 500.0, 40.0]
    m = oracle.OracleModel(c)
    assert [m.kbot(i, 0) for i in range(nx)] == [0, 1, 3, 4, 4]
    # u-faces are wet where both neighbouring cells are: Hu is the wet thickness
    Hu = m.get("Hu")[0]
    assert list(Hu[1:]) == [3000.0, 1000.0, 0.0, 0.0]
    assert Hu[0] == 0.0


def test_nonfinite_state_is_flagged():
    c = flat_box(4, 4, 3)
    m = oracle.OracleModel(c)
    assert not m.diagnostics()["nonfinite"]
    T = m.get("T")
    T[1, 2, 2] = np.nan
    m.set("T", T)
    assert m.diagnostics()["nonfinite"]
