"""Small hand-built cases used by the oracle pins and the GPU parity tests."""
from __future__ import annotations

import numpy as np

from paper_2309_06662_gb300 import inputs


def flat_box(nx, ny, nz, L=1.0e6, H=4000.0, periodic_x=False, periodic_y=False, T=None,
             S=None, u=None, v=None, eta=None, taux=None, tauy=None, **params) -> inputs.Case:
    """Flat-bottomed Cartesian box with uniform levels and the given state."""
    zf = inputs.uniform_z_faces(nz, H)
    depth = np.full((ny, nx), H)
    z = lambda val: np.zeros((nz, ny, nx)) + (0.0 if val is None else val)
    p = inputs.default_params()
    p.update(params)
    c = inputs.Case("flat_box", 0, nx, ny, nz, periodic_x, periodic_y, 0.0, L, 0.0, L, zf, depth,
                    np.zeros((ny, nx)) if taux is None else taux,
                    np.zeros((ny, nx)) if tauy is None else tauy,
                    z(10.0) if T is None else np.asarray(T, dtype=float) + np.zeros((nz, ny, nx)),
                    z(35.0) if S is None else np.asarray(S, dtype=float) + np.zeros((nz, ny, nx)),
                    p, steps=10)
    c.u = None if u is None else np.asarray(u, dtype=float) + np.zeros((nz, ny, nx))
    c.v = None if v is None else np.asarray(v, dtype=float) + np.zeros((nz, ny, nx))
    c.eta = None if eta is None else np.asarray(eta, dtype=float) + np.zeros((ny, nx))
    return c


NO_MIXING = dict(nu0=0.0, nu_b=0.0, kappa_b=0.0, kappa_conv=0.0)


def lake_at_rest(nx=48, ny=30, nz=10, seed=11) -> inputs.Case:
    """Seeded random-field bathymetry; T, S functions of depth only; no wind, no mixing."""
    c = inputs.latlon_case(nx, ny, nz, 70.0, seed, 1800.0, 20, 50, "lake", noise=0.0,
                           corr_deg=20.0)
    c = c.with_params(**NO_MIXING)
    c.taux[:] = 0.0
    c.tauy[:] = 0.0
    return c


def seeded_velocity(case: inputs.Case, seed: int, amp: float = 0.1):
    """Seeded smooth-ish random u, v fields (dry faces are zeroed by set_field)."""
    n = case.cells
    u = amp * inputs.random_normal(seed, 21, n).reshape(case.nz, case.ny, case.nx)
    v = amp * inputs.random_normal(seed, 22, n).reshape(case.nz, case.ny, case.nx)
    return u, v


def flat_latlon(nx, ny, nz, lat0=-60.0, lat1=60.0, H=4000.0, z_faces=None, T=None, S=None,
                u=None, v=None, eta=None, taux=None, tauy=None, **params) -> inputs.Case:
    """Flat-bottomed lat-lon band, periodic in longitude over 360 degrees, walls beyond
    the first and last rows; uniform levels unless z_faces is given."""
    zf = inputs.uniform_z_faces(nz, H) if z_faces is None else np.asarray(z_faces, dtype=float)
    depth = np.full((ny, nx), -zf[0])
    z = lambda val, d: np.zeros((nz, ny, nx)) + (d if val is None else np.asarray(val, dtype=float))
    p = inputs.default_params()
    p.update(params)
    c = inputs.Case("flat_latlon", 1, nx, ny, nz, True, False, 0.0, 360.0, lat0, lat1, zf,
                    depth, np.zeros((ny, nx)) if taux is None else taux,
                    np.zeros((ny, nx)) if tauy is None else tauy, z(T, 10.0), z(S, 35.0), p,
                    steps=10)
    c.u = None if u is None else z(u, 0.0)
    c.v = None if v is None else z(v, 0.0)
    c.eta = None if eta is None else np.asarray(eta, dtype=float) + np.zeros((ny, nx))
    return c
