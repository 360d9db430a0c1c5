"""Seeded synthetic inputs for the hydrostatic free-surface ocean step.

This module is shared by the CUDA library's tests and benchmark and by the CPU
oracle's tests.  It holds none of the method's arithmetic: it only places the
vertical levels, draws the random-field bathymetry, evaluates the surface wind
stress and the initial temperature/salinity fields, and collects the run
parameters.  Every random number comes from one counter-based generator
(SplitMix64, Steele, Lea & Flood 2014) followed by the Box-Muller transform, so
the same seed gives the same arrays on every machine.

The paper (Sec. "How performance was measured") forces its realistic domains with
ECCO2 fields over real bathymetry; neither is available here, so the recipes
below are synthetic stand-ins with the same shapes, depth range and forcing
magnitude.
"""
from __future__ import annotations

import math
import os
from dataclasses import dataclass, field, replace
from typing import Dict, Optional

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_STREAM = np.uint64(0xD1B54A32D192ED03)


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function applied elementwise to uint64 words."""
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def random_u64(seed: int, stream: int, start: int, n: int) -> np.ndarray:
    """Words start..start+n-1 of the SplitMix64 sequence keyed by (seed, stream)."""
    with np.errstate(over="ignore"):
        key = _mix64(np.array([np.uint64(seed) ^ (np.uint64(stream) * _STREAM)],
                              dtype=np.uint64))[0]
        ctr = np.arange(start + 1, start + n + 1, dtype=np.uint64)
        return _mix64(key + ctr * _GAMMA)


def random_normal(seed: int, stream: int, n: int, start: int = 0) -> np.ndarray:
    """n standard normal draws (Box-Muller on consecutive word pairs)."""
    with np.errstate(over="ignore"):
        w = random_u64(seed, stream, 2 * start, 2 * n).reshape(n, 2)
    u1 = ((w[:, 0] >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)
    u2 = (w[:, 1] >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


def random_uniform(seed: int, stream: int, n: int) -> np.ndarray:
    """n uniform draws in [0, 1)."""
    w = random_u64(seed, stream, 0, n)
    return (w >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


# ----------------------------------------------------------------------------- levels

def uniform_z_faces(nz: int, depth: float) -> np.ndarray:
    """nz+1 level faces from -depth (bottom) to 0 (top), evenly spaced."""
    return np.linspace(-depth, 0.0, nz + 1)


def stretched_z_faces(nz: int, depth: float = 5000.0, stretch: float = 3.0) -> np.ndarray:
    """nz+1 faces, bottom to top, thin near the surface.

    Face m below the surface sits at depth d(m) = H (exp(s m/nz) - 1)/(exp(s) - 1).
    """
    m = np.arange(nz + 1, dtype=np.float64)
    d = depth * (np.exp(stretch * m / nz) - 1.0) / (math.exp(stretch) - 1.0)
    d[-1] = depth
    return -d[::-1].copy()


# ----------------------------------------------------------------------------- bathymetry

def _gauss_filter_periodic(a: np.ndarray, sigma: float, axis: int) -> np.ndarray:
    n = a.shape[axis]
    k = np.fft.fftfreq(n) * 2.0 * math.pi
    h = np.exp(-0.5 * (sigma * k) ** 2)
    shape = [1] * a.ndim
    shape[axis] = n
    return np.real(np.fft.ifft(np.fft.fft(a, axis=axis) * h.reshape(shape), axis=axis))


def _gauss_filter_reflect(a: np.ndarray, sigma: float, axis: int) -> np.ndarray:
    n = a.shape[axis]
    b = np.concatenate([a, np.flip(a, axis=axis)], axis=axis)   # even extension
    b = _gauss_filter_periodic(b, sigma, axis)
    return np.take(b, np.arange(n), axis=axis)


def random_field_depth(nx: int, ny: int, dx_deg: float, dy_deg: float, seed: int,
                       corr_deg: float = 10.0, max_depth: float = 5500.0,
                       min_depth: float = 50.0, periodic_x: bool = True,
                       walls_y: bool = True) -> np.ndarray:
    """Seeded Gaussian random-field bathymetry (depth >= 0, metres), [ny, nx].

    White N(0,1) noise is smoothed by a Gaussian of standard deviation corr_deg
    (periodic in x when the domain is periodic, reflecting otherwise), min-max
    normalised to [0, max_depth]; columns shallower than min_depth become land
    (depth 0), and with walls_y the first and last rows are land.
    """
    noise = random_normal(seed, 1, nx * ny).reshape(ny, nx)
    f = noise
    if periodic_x:
        f = _gauss_filter_periodic(f, corr_deg / dx_deg, axis=1)
    else:
        f = _gauss_filter_reflect(f, corr_deg / dx_deg, axis=1)
    f = _gauss_filter_reflect(f, corr_deg / dy_deg, axis=0)
    f = (f - f.min()) / (f.max() - f.min())
    d = f * max_depth
    d[d < min_depth] = 0.0
    if walls_y:
        d[0, :] = 0.0
        d[-1, :] = 0.0
    return d


# ----------------------------------------------------------------------------- parameters

def default_params() -> Dict[str, float]:
    """Physical constants and scheme switches (the readings of the paper's unnamed constants)."""
    return dict(
        dt=600.0, n_substeps=30, chi=0.1,
        g=9.80665, rho0=1026.0, alpha=2e-4, beta_s=8e-4, T0=10.0, S0=35.0,
        f0=1e-4, beta_plane=2e-11, omega=7.292115e-5, radius=6.371e6,
        nu0=1e-2, ri_a=5.0, nu_b=1e-4, kappa_b=1e-5, kappa_conv=0.1,
        weno_eps=1e-30, weno_linear=0, min_depth=50.0, baro_filter=0,
        vertical_weno=0, momentum_vadv=0,
    )


@dataclass
class Case:
    """A complete seeded initial-value problem: grid, bathymetry, forcing, state, params."""
    name: str
    kind: int                 # 0 = Cartesian beta-plane box (metres), 1 = lat-lon (degrees)
    nx: int
    ny: int
    nz: int
    periodic_x: bool
    periodic_y: bool
    x0: float
    x1: float
    y0: float
    y1: float
    z_faces: np.ndarray       # nz+1, bottom to top
    depth: np.ndarray         # [ny, nx], metres, >= 0
    taux: np.ndarray          # [ny, nx] on u-faces, N/m^2
    tauy: np.ndarray          # [ny, nx] on v-faces, N/m^2
    T: np.ndarray             # [nz, ny, nx]
    S: np.ndarray             # [nz, ny, nx]
    params: Dict[str, float] = field(default_factory=default_params)
    steps: int = 100
    u: Optional[np.ndarray] = None
    v: Optional[np.ndarray] = None
    eta: Optional[np.ndarray] = None

    @property
    def cells(self) -> int:
        """Grid cells, land included."""
        return self.nx * self.ny * self.nz

    def with_params(self, **kw) -> "Case":
        """A copy of the case with some model parameters replaced."""
        p = dict(self.params)
        p.update(kw)
        return replace(self, params=p)


def _zc(zf: np.ndarray) -> np.ndarray:
    return 0.5 * (zf[1:] + zf[:-1])


def _noise_on_grid(seed: int, stream: int, level: int, ny: int, nx: int, lon0: float,
                   dlon: float, lat0: float, dlat: float, noise_deg: Optional[float],
                   periodic_x: bool) -> np.ndarray:
    """N(0,1) noise for one level.  With noise_deg, the draws sit on a noise_deg grid
    (periodic in longitude) and are interpolated bilinearly to the cell centres, which
    gives them a correlation length of about noise_deg; without, one draw per cell."""
    if noise_deg is None:
        return random_normal(seed, stream, ny * nx, start=level * ny * nx).reshape(ny, nx)
    nxc = max(1, int(round(nx * dlon / noise_deg)))
    nyc = max(2, int(round(ny * dlat / noise_deg)) + 1)
    base = random_normal(seed, stream, nyc * nxc, start=level * nyc * nxc).reshape(nyc, nxc)
    fy = (lat0 + (np.arange(ny) + 0.5) * dlat - lat0) / noise_deg - 0.5
    fy = np.clip(fy, 0.0, nyc - 1.0)
    jy0 = np.minimum(np.floor(fy).astype(int), nyc - 2)
    wy = (fy - jy0)[:, None]
    rows = (1.0 - wy) * base[jy0] + wy * base[jy0 + 1]
    fx = ((np.arange(nx) + 0.5) * dlon) / noise_deg - 0.5
    ix0 = np.floor(fx).astype(int)
    wx = (fx - ix0)[None, :]
    if periodic_x:
        i0, i1 = ix0 % nxc, (ix0 + 1) % nxc
    else:
        i0, i1 = np.clip(ix0, 0, nxc - 1), np.clip(ix0 + 1, 0, nxc - 1)
    return (1.0 - wx) * rows[:, i0] + wx * rows[:, i1]


def _stratified(zf: np.ndarray, ny: int, nx: int, seed: int, t_top: float, t_bot: float,
                s_top: float, s_bot: float, noise: float, grid=None,
                noise_deg: Optional[float] = None) -> tuple:
    """T and S linear in depth (top and bottom values) plus `noise` times N(0,1) noise.
    `grid` = (lon0, dlon, lat0, dlat, periodic_x) places the noise for noise_deg."""
    nz = len(zf) - 1
    H = -zf[0]
    zc = _zc(zf)
    frac = (zc + H) / H                      # 0 at the bottom, 1 at the top
    T = np.empty((nz, ny, nx))
    S = np.empty((nz, ny, nx))
    lon0, dlon, lat0, dlat, px = grid if grid is not None else (0.0, 1.0, 0.0, 1.0, True)

    def level(k):
        T[k] = t_bot + (t_top - t_bot) * frac[k]
        S[k] = s_bot + (s_top - s_bot) * frac[k]
        if noise > 0:
            T[k] += noise * _noise_on_grid(seed, 2, k, ny, nx, lon0, dlon, lat0, dlat,
                                           noise_deg, px)
            if s_top != s_bot:
                S[k] += noise * _noise_on_grid(seed, 3, k, ny, nx, lon0, dlon, lat0, dlat,
                                               noise_deg, px)

    if ny * nx * nz >= 1 << 22:      # large grids: levels in parallel (numpy releases the GIL)
        from concurrent.futures import ThreadPoolExecutor
        with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
            list(ex.map(level, range(nz)))
    else:
        for k in range(nz):
            level(k)
    return T, S


def box_case(nx: int = 32, ny: int = 32, nz: int = 8, seed: int = 1) -> Case:
    """Closed 1000 km x 1000 km beta-plane box, flat 4 km bottom, double-gyre wind.

    T is linear from 20 C (top) to 2 C (bottom) plus N(0, 0.01 C) noise; S = 35.
    """
    L = 1.0e6
    zf = uniform_z_faces(nz, 4000.0)
    depth = np.full((ny, nx), 4000.0)
    yc = (np.arange(ny) + 0.5) * (L / ny)
    taux = np.repeat((0.1 * np.cos(math.pi * yc / L))[:, None], nx, axis=1)
    tauy = np.zeros((ny, nx))
    T, S = _stratified(zf, ny, nx, seed, 20.0, 2.0, 35.0, 35.0, 0.01)
    p = default_params()
    p.update(dt=600.0, n_substeps=30)
    return Case("box", 0, nx, ny, nz, False, False, 0.0, L, 0.0, L, zf, depth, taux, tauy,
                T, S, p, steps=100)


def latlon_case(nx: int, ny: int, nz: int, lat: float, seed: int, dt: float, n_substeps: int,
                steps: int, name: str, noise: float = 0.05, corr_deg: float = 10.0,
                noise_deg: Optional[float] = 1.0) -> Case:
    """Global lat-lon channel from -lat to +lat, periodic in longitude, walls at both ends.

    Stretched levels to 5000 m, random-field bathymetry, zonal wind 0.1 cos(3 phi) N/m^2,
    T linear 20 -> 2 C and S linear 34.5 -> 35 with depth, each with `noise`-amplitude
    N(0,1) perturbations drawn on a noise_deg grid (1 degree: one draw per cell of the
    1-degree grid, a mesoscale correlation length on finer grids).
    """
    zf = stretched_z_faces(nz, 5000.0, 3.0)
    dlon = 360.0 / nx
    dlat = 2.0 * lat / ny
    depth = random_field_depth(nx, ny, dlon, dlat, seed, corr_deg=corr_deg)
    phi = np.deg2rad(-lat + (np.arange(ny) + 0.5) * dlat)
    taux = np.repeat((0.1 * np.cos(3.0 * phi))[:, None], nx, axis=1)
    tauy = np.zeros((ny, nx))
    T, S = _stratified(zf, ny, nx, seed, 20.0, 2.0, 34.5, 35.0, noise,
                       grid=(0.0, dlon, -lat, dlat, True), noise_deg=noise_deg)
    p = default_params()
    p.update(dt=dt, n_substeps=n_substeps)
    return Case(name, 1, nx, ny, nz, True, False, 0.0, 360.0, -lat, lat, zf, depth, taux,
                tauy, T, S, p, steps=steps)


def latlon_1deg_case(seed: int = 2) -> Case:
    """1-degree, 360 x 160 x 32, 80S-80N, dt = 1200 s, 40 substeps, 1000 steps."""
    return latlon_case(360, 160, 32, 80.0, seed, 1200.0, 40, 1000, "latlon_1deg")


def latlon_12th_case(seed: int = 3, dt: float = 180.0) -> Case:
    """1/12-degree, 4320 x 1680 x 48, 70S-70N, 60 substeps, 200 steps.

    dt = 180 s, the paper's own step for its 1/12-degree, 48-level run (table of GPU
    model performance).  At 300 s the explicit quasi-AB2 step is past its internal
    gravity-wave limit next to 70 degrees (dx = 3.2 km, first-mode speed ~4.4 m/s with
    this stratification: omega dt ~ 0.88 for the shortest waves, while chi = 0.1 damps
    only below ~0.63) and the state diverges within about 30 steps."""
    return latlon_case(4320, 1680, 48, 70.0, seed, dt, 60, 200, "latlon_12th")


def latlon_quarter_case(seed: int = 6) -> Case:
    """1/4-degree, 1440 x 560 x 48, 70S-70N, dt = 900 s, 60 substeps (a profiling-size
    member of the same recipe: every 3-D FP32 field is larger than L2)."""
    return latlon_case(1440, 560, 48, 70.0, seed, 900.0, 60, 200, "latlon_quarter")


def latlon_half_case(seed: int = 4, lat: float = 80.0) -> Case:
    """1/2-degree, 720 x 320 x 48, 80S-80N, dt = 480 s (the step of the coarse model of the
    closure experiments), 60 substeps, 2000 steps."""
    return latlon_case(720, 320, 48, lat, seed, 480.0, 60, 2000, "latlon_half")


def latlon_half70_case(seed: int = 3) -> Case:
    """1/2-degree restriction of the 1/12-degree recipe: 720 x 280 x 48, 70S-70N, the same
    seeded random-field bathymetry and forcing recipe generated at 1/2 degree, dt = 480 s
    (the 1/2-degree step of this recipe, below the internal-wave limit next to 70 degrees),
    60 substeps, 200 steps; the size at which the oracle runs the recipe."""
    return latlon_case(720, 280, 48, 70.0, seed, 480.0, 60, 200, "latlon_half70")


def aquaplanet_case(nx: int = 2160, ny: int = 900, nz: int = 100, seed: int = 8,
                    dt: float = 240.0, n_substeps: int = 30, depth: float = 4000.0,
                    ridge_deg: float = 1.0) -> Case:
    """The per-GPU workload of the paper's aqua-planet weak-scaling runs (Sec. "How
    performance was measured": global, 75S-75N, 100 levels, idealised bathymetry with two
    ridges that divide the world ocean into two basins; each GPU holds the equivalent of a
    global 1/6-degree grid).  The ridge geometry is not given; here: a flat 4000 m ocean
    with two land ridges `ridge_deg` wide at 0 and 90 degrees east, from the northern edge
    down to 35S, so that the basins meet in a circumpolar channel south of 35S.  Stretched
    levels, zonal wind 0.1 cos(3 phi) N/m^2, T linear 20 -> 2 C in depth scaled towards
    the poles by cos(phi) (cold high latitudes) plus 0.05 C of seeded noise, S 34.5 -> 35;
    dt = 240 s (below the internal-wave limit of the 4.8 km zonal spacing at 75 degrees),
    30 substeps, 500 steps (the paper's averaging window)."""
    lat = 75.0
    zf = stretched_z_faces(nz, depth, 3.0)
    dlon, dlat = 360.0 / nx, 2.0 * lat / ny
    lonc = (np.arange(nx) + 0.5) * dlon
    latc = -lat + (np.arange(ny) + 0.5) * dlat
    d = np.full((ny, nx), depth)
    for lon0 in (0.0, 90.0):
        dl = np.abs((lonc - lon0 + 180.0) % 360.0 - 180.0)
        ridge = dl <= max(0.5 * ridge_deg, 0.5 * dlon)   # at least the nearest cells
        d[np.ix_(latc > -35.0, ridge)] = 0.0
    phi = np.deg2rad(latc)
    taux = np.repeat((0.1 * np.cos(3.0 * phi))[:, None], nx, axis=1)
    tauy = np.zeros((ny, nx))
    T, S = _stratified(zf, ny, nx, seed, 20.0, 2.0, 34.5, 35.0, 0.05,
                       grid=(0.0, dlon, -lat, dlat, True), noise_deg=1.0)
    # warm low latitudes, cold high latitudes: the top-to-bottom contrast shrinks with
    # cos(phi) toward the poles (the deep value stays at 2 C)
    T = 2.0 + (T - 2.0) * np.cos(phi)[None, :, None]
    p = default_params()
    p.update(dt=dt, n_substeps=n_substeps)
    return Case("aquaplanet", 1, nx, ny, nz, True, False, 0.0, 360.0, -lat, lat, zf, d, taux,
                tauy, T, S, p, steps=500)


def latlon_small_case(nx: int = 72, ny: int = 40, nz: int = 12, seed: int = 7,
                      lat: float = 70.0, dt: float = 1800.0, n_substeps: int = 20) -> Case:
    """A small lat-lon case (5 degree) with the same recipe, for fast parity runs."""
    return latlon_case(nx, ny, nz, lat, seed, dt, n_substeps, 50, "latlon_small",
                       corr_deg=20.0)


def latlon_window(case_nx: int, case_ny: int, lat: float, i0: int, j0: int, wx: int,
                  wy: int) -> tuple:
    """Lon/lat bounds of the sub-window [i0, i0+wx) x [j0, j0+wy) of a global lat-lon grid."""
    dlon = 360.0 / case_nx
    dlat = 2.0 * lat / case_ny
    return (i0 * dlon, (i0 + wx) * dlon, -lat + j0 * dlat, -lat + (j0 + wy) * dlat)


def latlon_window_case(case: Case, i0: int, j0: int, wx: int, wy: int) -> Case:
    """The sub-window [i0, i0+wx) x [j0, j0+wy) of a lat-lon case as a closed basin
    (walls at its edges): same metrics, levels, bathymetry, forcing, state, parameters."""
    x0, x1, y0, y1 = latlon_window(case.nx, case.ny, case.y1, i0, j0, wx, wy)
    sl = (slice(j0, j0 + wy), slice(i0, i0 + wx))
    cut3 = lambda F: None if F is None else F[(slice(None),) + sl].copy()
    return Case(f"{case.name}_window", case.kind, wx, wy, case.nz, False, False, x0, x1, y0,
                y1, case.z_faces, case.depth[sl].copy(), case.taux[sl].copy(),
                case.tauy[sl].copy(), cut3(case.T), cut3(case.S), dict(case.params),
                steps=case.steps, u=cut3(case.u), v=cut3(case.v),
                eta=None if case.eta is None else case.eta[sl].copy())


# ----------------------------------------------------------------------------- closure weights

def mlp_seeded_params(seed: int, dims, gain: float = 1.0):
    """Seeded initial weights of a column MLP with layer widths `dims`: W [in, out] and b
    [out] per layer, drawn N(0, gain^2/in) and stored as integers |n| <= 255 times a power
    of two, so every value is exactly representable in bfloat16 (and float32)."""
    params = []
    for li, (a, b) in enumerate(zip(dims[:-1], dims[1:])):
        sigma = gain / math.sqrt(a)
        q = 6 - int(math.floor(math.log2(sigma)))          # sigma * 2^q in [64, 128)
        n = np.clip(np.round(random_normal(seed, 100 + li, a * b) * sigma * 2.0 ** q), -255, 255)
        W = (n * 2.0 ** -q).reshape(a, b)
        nb = np.clip(np.round(random_normal(seed, 200 + li, b) * 0.1 * sigma * 2.0 ** q), -255, 255)
        params.append((W, nb * 2.0 ** -q))
    return params


def restrict_depth(depth: np.ndarray, r: int, row_area: np.ndarray,
                   min_depth: float = 50.0) -> np.ndarray:
    """Coarse bathymetry of r x r blocks: area-weighted mean depth (land counting as 0),
    columns shallower than min_depth become land."""
    ny, nx = depth.shape
    a = np.broadcast_to(row_area[:, None], (ny, nx))
    d = (depth * a).reshape(ny // r, r, nx // r, r).sum(axis=(1, 3))
    d /= a.reshape(ny // r, r, nx // r, r).sum(axis=(1, 3))
    d[d < min_depth] = 0.0
    return d


def latlon_row_area(ny: int, lat: float, nx: int, radius: float = 6.371e6) -> np.ndarray:
    """Cell area per row of a global lat-lon grid from -lat to lat (the product form
    R cos(phi) dlambda R dphi)."""
    dphi = math.radians(2.0 * lat / ny)
    phi = np.radians(-lat + (np.arange(ny) + 0.5) * (2.0 * lat / ny))
    return radius * np.cos(phi) * math.radians(360.0 / nx) * radius * dphi


def latlon_pair(nxc: int, nyc: int, nz: int, lat: float, r: int, seed: int, dt_coarse: float,
                ns_coarse: int, ns_fine: int, corr_deg: float = 10.0, noise: float = 0.05):
    """A fine lat-lon case (r times finer, dt/r) and its coarse counterpart whose
    bathymetry is the fine one restricted to r x r blocks; the coarse T, S start as block
    means of the fine ones."""
    fine = latlon_case(r * nxc, r * nyc, nz, lat, seed, dt_coarse / r, ns_fine, 1, "fine",
                       noise=noise, corr_deg=corr_deg)
    area = latlon_row_area(r * nyc, lat, r * nxc)
    dc = restrict_depth(fine.depth, r, area)
    dc[0, :] = 0.0
    dc[-1, :] = 0.0
    blk = lambda F: F.reshape(nz, nyc, r, nxc, r).mean(axis=(2, 4))
    coarse = Case("coarse", 1, nxc, nyc, nz, True, False, 0.0, 360.0, -lat, lat, fine.z_faces, dc,
                  fine.taux.reshape(nyc, r, nxc, r).mean(axis=(1, 3)),
                  np.zeros((nyc, nxc)), blk(fine.T), blk(fine.S), dict(fine.params), steps=1)
    coarse.params["dt"] = dt_coarse
    coarse.params["n_substeps"] = ns_coarse
    return fine, coarse


# ----------------------------------------------------------------------------- ensemble

def ensemble_member_case(seed: int, nx: int, ny: int, nz: int, wind: float, dT: float,
                         dx: float = 20e3) -> Case:
    """One closed beta-plane basin of the ensemble: dx = dy = 20 km, uniform levels to
    5500 m, random-field bathymetry (correlation 10 cells, land where shallower than
    50 m and on the first and last rows), zonal wind `wind` cos(pi y / Ly), T linear
    from 2 + dT (top) to 2 C and S from 34.5 to 35 with 0.05 noise, dt 600 s, 30
    substeps."""
    zf = uniform_z_faces(nz, 5500.0)
    depth = random_field_depth(nx, ny, 1.0, 1.0, seed, corr_deg=10.0, periodic_x=False)
    Ly = ny * dx
    yc = (np.arange(ny) + 0.5) * dx
    taux = np.repeat((wind * np.cos(math.pi * yc / Ly))[:, None], nx, axis=1)
    tauy = np.zeros((ny, nx))
    T, S = _stratified(zf, ny, nx, seed, 2.0 + dT, 2.0, 34.5, 35.0, 0.05)
    p = default_params()
    p.update(dt=600.0, n_substeps=30)
    return Case(f"member_{seed}", 0, nx, ny, nz, False, False, 0.0, nx * dx, 0.0, Ly, zf,
                depth, taux, tauy, T, S, p, steps=1)


def ensemble_cases(count: int = 96, seed: int = 5, n_lo: int = 32, n_hi: int = 512,
                   levels=(8, 16, 32, 48)):
    """`count` uneven members: member m draws (seed + m) nx, ny ~ U[n_lo, n_hi], nz from
    `levels`, wind ~ U[0.05, 0.2] N/m^2 and dT ~ U[10, 20] C."""
    out = []
    for m in range(count):
        s = seed + m
        u = random_uniform(s, 50, 5)
        nx = n_lo + int(u[0] * (n_hi - n_lo + 1))
        ny = n_lo + int(u[1] * (n_hi - n_lo + 1))
        nz = int(levels[int(u[2] * len(levels))])
        out.append(ensemble_member_case(s, nx, ny, nz, 0.05 + 0.15 * u[3], 10.0 + 10.0 * u[4]))
    return out


# the benchmark's workloads: name -> (case constructor, workload label)
WORKLOADS = {
    "latlon_12th": (latlon_12th_case, "latlon_1/12deg_4320x1680x48"),
    "latlon_quarter": (latlon_quarter_case, "latlon_1/4deg_1440x560x48"),
    "latlon_1deg": (latlon_1deg_case, "latlon_1deg_360x160x32"),
    "box": (box_case, "box_32x32x8"),
    "ensemble96": (lambda: ensemble_cases(96, seed=5), "ensemble_96_basins"),
    "learned_half": (latlon_half_case, "latlon_1/2deg_720x320x48_learned_closure"),
    "aquaplanet_6th": (aquaplanet_case, "aquaplanet_1/6deg_2160x900x100"),
}
