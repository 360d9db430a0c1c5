"""The C-ABI library builds for sm_103a, loads without a GPU and exports every symbol
the public headers declare (no compute calls here)."""
import ctypes
import glob
import os
import re

from paper_2309_06662_gb300 import build, ocean

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"\b([a-z][a-z0-9_]+)\s*\([^;{]*\)\s*;", txt))
    return sorted(n for n in names if not n.startswith(("sizeof", "if", "for")))


def test_library_exports_every_declared_function():
    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert "ocean_step" in names and "ocean_create" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_header():
    L = ocean.load()
    for n in ocean.header_functions():
        assert getattr(L, n).argtypes is not None, n


def test_arena_size_and_argument_errors_without_gpu():
    # host-side validation paths run without touching a device
    from paper_2309_06662_gb300 import inputs
    c = inputs.box_case()
    L = ocean.load()
    g, _zf = ocean.make_grid(c)
    prm, _keep = ocean.make_params(c.params, ocean.OCEAN_MIXED, c.taux, c.tauy)
    nb = ctypes.c_size_t()
    assert L.ocean_arena_bytes(ctypes.byref(g), ctypes.byref(prm), ctypes.byref(nb)) == 0
    assert nb.value > 16 * 32 * 32 * 8 * 4
    prm64, _k = ocean.make_params(c.params, ocean.OCEAN_FP64, c.taux, c.tauy)
    nb64 = ctypes.c_size_t()
    L.ocean_arena_bytes(ctypes.byref(g), ctypes.byref(prm64), ctypes.byref(nb64))
    assert nb64.value > nb.value
    bad = ocean.OceanGrid(0, 0, 4, 4, 0, 0, 0.0, 1.0, 0.0, 1.0, g.z_faces)
    assert L.ocean_arena_bytes(ctypes.byref(bad), ctypes.byref(prm), ctypes.byref(nb)) == -1
    assert b"grid sizes" in L.ocean_last_error(None)
    prm.n_substeps = 0
    assert L.ocean_arena_bytes(ctypes.byref(g), ctypes.byref(prm), ctypes.byref(nb)) == -1
    prm.n_substeps = 30
    # a padded 3-D array of 2^31 cells or more is refused (32-bit cell offsets): 30000 x
    # 30000 columns pass the column limit, 30000 x 30000 x 8 cells do not
    huge = ocean.OceanGrid(g.kind, 30000, 30000, g.nz, 0, 0, 0.0, 1.0, 0.0, 1.0, g.z_faces)
    assert L.ocean_arena_bytes(ctypes.byref(huge), ctypes.byref(prm), ctypes.byref(nb)) == -1
    assert b"2^31" in L.ocean_last_error(None)
    prm.n_substeps = 30
    h = ctypes.c_void_p()
    assert L.ocean_create(ctypes.byref(g), None, ctypes.byref(prm), ctypes.byref(h)) == -1
    assert L.ocean_step(None, 1) == -1
    assert L.ocean_get_step(None) == -1
    assert L.ocean_set_wind_stress(None, None, None) == -1
    assert L.ocean_set_wind_stress_f32(None, None, None) == -1
    assert b"null handle" in L.ocean_last_error(None)


def test_ensemble_argument_errors_without_gpu():
    # ocean_ensemble_create checks its members on the host before any device call
    from paper_2309_06662_gb300 import inputs
    cases = inputs.ensemble_cases(2, seed=60, n_lo=8, n_hi=12, levels=(4,))
    L = ocean.load()
    M = len(cases)
    grids = (ocean.OceanGrid * M)()
    prms = (ocean.OceanParams * M)()
    depths = (ctypes.POINTER(ctypes.c_double) * M)()
    keep = []
    for i, c in enumerate(cases):
        g, zf = ocean.make_grid(c)
        p, k = ocean.make_params(c.params, ocean.OCEAN_MIXED, c.taux, c.tauy)
        import numpy as np
        d = np.ascontiguousarray(c.depth)
        keep += [zf, k, d]
        grids[i], prms[i] = g, p
        depths[i] = d.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    h = ctypes.c_void_p()
    grids[1].periodic_x = 1
    assert L.ocean_ensemble_create(M, grids, depths, prms, ctypes.byref(h)) == -1
    assert b"closed basins" in L.ocean_last_error(None)
    grids[1].periodic_x = 0
    prms[1].dt = 300.0
    assert L.ocean_ensemble_create(M, grids, depths, prms, ctypes.byref(h)) == -1
    assert b"share precision" in L.ocean_last_error(None)
    prms[1].dt = prms[0].dt
    prms[0].closure = ocean.OCEAN_CLOSURE_LEARNED
    assert L.ocean_ensemble_create(M, grids, depths, prms, ctypes.byref(h)) == -1
    prms[0].closure = ocean.OCEAN_CLOSURE_RI
    assert L.ocean_ensemble_create(0, grids, depths, prms, ctypes.byref(h)) == -1
    assert L.ocean_ensemble_step(None, 1) == -1
    assert L.ocean_ensemble_member(None, 0) is None
    assert L.ocean_ensemble_kernel_launches(None) == -1


def test_ensemble_recipe():
    from paper_2309_06662_gb300 import inputs
    cs = inputs.ensemble_cases(12, seed=5)
    for c in cs:
        assert 32 <= c.nx <= 512 and 32 <= c.ny <= 512 and c.nz in (8, 16, 32, 48)
        assert not c.periodic_x and not c.periodic_y and c.kind == 0
        assert c.depth.max() <= 5500.0 and (c.depth[0] == 0).all() and (c.depth[-1] == 0).all()
        assert 0.05 <= c.taux.max() <= 0.2 + 1e-12
        assert c.params["dt"] == 600.0 and c.params["n_substeps"] == 30
    assert len({(c.nx, c.ny, c.nz) for c in cs}) == len(cs)     # uneven members
    again = inputs.ensemble_cases(12, seed=5)
    assert all((a.depth == b.depth).all() and (a.T == b.T).all() for a, b in zip(cs, again))
