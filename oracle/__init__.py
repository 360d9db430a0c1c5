"""Plain FP64 CPU oracle of the ocean step (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and its
Python binding) never touches it.  The C source, ``ocean_oracle.c``, states the
discrete equations it follows; this wrapper only builds and marshals.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Dict, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ocean_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

FIELD_IDS = dict(u=0, v=1, T=2, S=3, eta=4, Gu_prev=5, Gv_prev=6, GT_prev=7, GS_prev=8,
                 w=9, p=10, kappa=11, nu=12, Gu=13, Gv=14, GT=15, GS=16, Hu=17, Hv=18, b=19)
FIELDS_2D = {"eta", "Hu", "Hv"}
PRM_ORDER = ["dt", "chi", "g", "rho0", "alpha", "beta_s", "T0", "S0", "f0", "beta_plane",
             "omega", "radius", "nu0", "ri_a", "nu_b", "kappa_b", "kappa_conv", "weno_eps",
             "min_depth"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no fast-math, no FMA contraction)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if (not force and os.path.exists(_OUT)
            and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC)):
        return _OUT
    tmp = _OUT + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _OUT)
    return _OUT


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            P = ctypes.POINTER
            d, i = ctypes.c_double, ctypes.c_int
            L.ora_create.restype = ctypes.c_void_p
            L.ora_create.argtypes = [P(i), P(d), P(d), P(d), P(d), P(d), P(d), P(i)]
            L.ora_destroy.argtypes = [ctypes.c_void_p]
            L.ora_step.argtypes = [ctypes.c_void_p, i]
            L.ora_tendencies.argtypes = [ctypes.c_void_p]
            L.ora_set_field.argtypes = [ctypes.c_void_p, i, P(d)]
            L.ora_get_field.argtypes = [ctypes.c_void_p, i, P(d)]
            L.ora_diagnostics.argtypes = [ctypes.c_void_p, P(d)]
            L.ora_get_step.restype = ctypes.c_long
            L.ora_get_step.argtypes = [ctypes.c_void_p]
            L.ora_set_step.argtypes = [ctypes.c_void_p, ctypes.c_long]
            L.ora_weno5.restype = d
            L.ora_weno5.argtypes = [P(d), d, i]
            L.ora_weno3.restype = d
            L.ora_weno3.argtypes = [P(d), d, i]
            L.ora_recon.restype = d
            L.ora_recon.argtypes = [P(d), P(i), d, i]
            L.ora_recon_coef.restype = d
            L.ora_recon_coef.argtypes = [P(d), P(i), P(d), d, d, i]
            L.ora_weno_coeffs.argtypes = [P(d), d, i, P(d)]
            L.ora_vertical_advection_column.argtypes = [i, P(d), P(d), i, P(d), i, i, d, P(d)]
            L.ora_thomas.argtypes = [i, P(d), P(d), P(d), P(d), P(d)]
            L.ora_barotropic.argtypes = [ctypes.c_void_p, P(d), P(d), P(d), P(d), P(d), P(d), P(d)]
            L.ora_set_closure_fields.argtypes = [ctypes.c_void_p, P(d), P(d), P(d)]
            L.ora_kbot.restype = i
            L.ora_filter_weights.restype = d
            L.ora_filter_weights.argtypes = [i, i, P(d)]
            L.ora_kbot.argtypes = [ctypes.c_void_p, i, i]
            L.ora_set_threads.argtypes = [i]
            L.ora_get_threads.restype = i
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def weno5(q, eps: float = 1e-30, linear: bool = False) -> float:
    q = _f64(q)
    return lib().ora_weno5(_dp(q), eps, int(linear))


def weno3(q, eps: float = 1e-30, linear: bool = False) -> float:
    q = _f64(q)
    return lib().ora_weno3(_dp(q), eps, int(linear))


def recon(q, inside, eps: float = 1e-30, linear: bool = False) -> float:
    q = _f64(q)
    ins = np.ascontiguousarray(inside, dtype=np.int32)
    return lib().ora_recon(_dp(q), ins.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), eps, int(linear))


def recon_coef(q, inside, edges, xf: float, eps: float = 1e-30, linear: bool = False) -> float:
    """Adaptive-order WENO-Z at xf of an ordered five-cell stencil with edges[0..5] (the
    candidates and ideal weights of that non-uniform stencil)."""
    q, e = _f64(q), _f64(edges)
    ins = np.ascontiguousarray(inside, dtype=np.int32)
    return lib().ora_recon_coef(_dp(q), ins.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(e),
                                float(xf), eps, int(linear))


def weno_coeffs(edges, xf: float, five: bool = True):
    """Stretched-stencil coefficients: (c [3][3], d [3], c3 [2][2], d3 [2])."""
    e = _f64(edges)
    out = np.zeros(18)
    lib().ora_weno_coeffs(_dp(e), float(xf), int(five), _dp(out))
    return out[:9].reshape(3, 3), out[9:12], out[12:16].reshape(2, 2), out[16:18]


def vertical_advection_column(z_faces, F, k0: int, w_faces, vertical_weno: int = 1,
                              momentum_vadv: int = 1, eps: float = 1e-30) -> np.ndarray:
    """w dF/dz of one velocity column as the momentum tendency computes it (levels k0..nz-1;
    w_faces[k] on the bottom face of level k, nz + 1 values)."""
    zf, F, wf = _f64(z_faces), _f64(F), _f64(w_faces)
    nz = len(F)
    out = np.zeros(nz)
    lib().ora_vertical_advection_column(nz, _dp(zf), _dp(F), int(k0), _dp(wf), int(vertical_weno),
                                        int(momentum_vadv), eps, _dp(out))
    return out


def set_threads(n: int) -> None:
    """Threads of the oracle's OpenMP row loops."""
    lib().ora_set_threads(int(n))


def get_threads() -> int:
    return int(lib().ora_get_threads())


def filter_weights(ns: int, kind: int = 0):
    """Averaging weights a_1..a_ns of the sub-cycle and their first moment sum m a_m."""
    a = np.zeros(ns)
    mom = lib().ora_filter_weights(int(ns), int(kind), _dp(a))
    return a, mom


def thomas(a, b, c, d) -> np.ndarray:
    a, b, c, d = (_f64(x) for x in (a, b, c, d))
    x = np.zeros_like(d)
    lib().ora_thomas(len(d), _dp(a), _dp(b), _dp(c), _dp(d), _dp(x))
    return x


class OracleModel:
    """One oracle model instance built from an ``inputs.Case``."""

    def __init__(self, case, params: Optional[Dict[str, float]] = None):
        p = dict(case.params)
        if params:
            p.update(params)
        self.case = case
        self.params = p
        self.nx, self.ny, self.nz = case.nx, case.ny, case.nz
        ig = np.array([case.kind, case.nx, case.ny, case.nz, int(case.periodic_x),
                       int(case.periodic_y)], dtype=np.int32)
        dg = _f64([case.x0, case.x1, case.y0, case.y1])
        prm = _f64([p[k] for k in PRM_ORDER])
        ip = np.array([int(p["n_substeps"]), int(p["weno_linear"]), int(p.get("baro_filter", 0)),
                       int(p.get("vertical_weno", 0)), int(p.get("momentum_vadv", 0))],
                      dtype=np.int32)
        keep = [_f64(case.z_faces), _f64(case.depth), _f64(case.taux), _f64(case.tauy)]
        L = lib()
        self._h = L.ora_create(ig.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(dg),
                               *(_dp(a) for a in keep), _dp(prm),
                               ip.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
        self.set("T", case.T)
        self.set("S", case.S)
        if case.u is not None:
            self.set("u", case.u)
        if case.v is not None:
            self.set("v", case.v)
        if case.eta is not None:
            self.set("eta", case.eta)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().ora_destroy(h)
            self._h = None

    def shape(self, name: str):
        return (self.ny, self.nx) if name in FIELDS_2D else (self.nz, self.ny, self.nx)

    def set(self, name: str, arr) -> None:
        a = _f64(arr)
        assert a.shape == self.shape(name), (name, a.shape)
        rc = lib().ora_set_field(self._h, FIELD_IDS[name], _dp(a))
        assert rc == 0

    def get(self, name: str) -> np.ndarray:
        out = np.zeros(self.shape(name))
        rc = lib().ora_get_field(self._h, FIELD_IDS[name], _dp(out))
        assert rc == 0
        return out

    def step(self, n: int = 1) -> None:
        lib().ora_step(self._h, int(n))

    def tendencies(self) -> None:
        lib().ora_tendencies(self._h)

    @property
    def nstep(self) -> int:
        return lib().ora_get_step(self._h)

    @nstep.setter
    def nstep(self, n: int) -> None:
        lib().ora_set_step(self._h, int(n))

    def kbot(self, i: int, j: int) -> int:
        return lib().ora_kbot(self._h, i, j)

    def diagnostics(self) -> Dict[str, float]:
        out = np.zeros(8)
        lib().ora_diagnostics(self._h, _dp(out))
        return dict(tracer_T=out[0], tracer_S=out[1], volume_eta=out[2], ke=out[3],
                    max_cfl=out[4], nonfinite=bool(out[5]), wet_volume=out[6], step=int(out[7]))

    def kb_array(self):
        return np.array([[self.kbot(i, j) for i in range(self.nx)] for j in range(self.ny)])

    def set_closure_fields(self, kappa, dGT, dGS) -> None:
        """Learned diffusivity and tracer corrections for the next steps (None: remove)."""
        if kappa is None:
            lib().ora_set_closure_fields(self._h, None, None, None)
            return
        k, a, b = (_f64(x) for x in (kappa, dGT, dGS))
        lib().ora_set_closure_fields(self._h, _dp(k), _dp(a), _dp(b))

    def barotropic(self, eta, U, V, GU, GV):
        """Run the sub-cycle alone; returns (eta_bar, U_bar, V_bar)."""
        e = _f64(eta).copy()
        U, V, GU, GV = (_f64(x) for x in (U, V, GU, GV))
        Ub = np.zeros_like(e)
        Vb = np.zeros_like(e)
        lib().ora_barotropic(self._h, _dp(e), _dp(U), _dp(V), _dp(GU), _dp(GV), _dp(Ub), _dp(Vb))
        return e, Ub, Vb
