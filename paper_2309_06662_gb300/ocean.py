"""Thin Python binding of libocean (include/ocean.h): argument marshalling only.

The functions below carry the C names and call straight into the CUDA library; every
step of the ocean model runs in its kernels.  PyTorch supplies device memory (the
arena passed to ocean_create_in) and the CUDA stream.  There is no CPU fallback: if
the library cannot be loaded, or no CUDA device is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading
from ctypes import POINTER, c_double, c_int, c_long, c_size_t, c_void_p
from typing import Dict, Optional

import numpy as np

from . import build as _build

OCEAN_OK = 0
OCEAN_ERR = {-1: "OCEAN_ERR_ARG", -2: "OCEAN_ERR_CUDA", -3: "OCEAN_ERR_NONFINITE",
             -4: "OCEAN_ERR_TIMEOUT", -5: "OCEAN_ERR_OOM", -6: "OCEAN_ERR_STATE"}
OCEAN_FP64, OCEAN_MIXED = 0, 1
OCEAN_CLOSURE_RI, OCEAN_CLOSURE_LEARNED = 0, 1

FIELD = dict(u=0, v=1, T=2, S=3, eta=4, Gu_prev=5, Gv_prev=6, GT_prev=7, GS_prev=8, w=9, p=10,
             kappa=11, nu=12, Gu=13, Gv=14, GT=15, GS=16, Hu=17, Hv=18, T_anom=19, S_anom=20)
# everything a bitwise restart needs, besides the reference profiles and the step count
CHECKPOINT_FIELDS = ["u", "v", "T_anom", "S_anom", "eta", "Gu_prev", "Gv_prev", "GT_prev",
                     "GS_prev"]
FIELDS_2D = {"eta", "Hu", "Hv"}

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                      "ocean.h")


class OceanGrid(ctypes.Structure):
    _fields_ = [("kind", c_int), ("nx", c_int), ("ny", c_int), ("nz", c_int),
                ("periodic_x", c_int), ("periodic_y", c_int), ("x0", c_double), ("x1", c_double),
                ("y0", c_double), ("y1", c_double), ("z_faces", POINTER(c_double))]


class OceanParams(ctypes.Structure):
    _fields_ = [("dt", c_double), ("n_substeps", c_int), ("chi", c_double), ("g", c_double),
                ("rho0", c_double), ("alpha", c_double), ("beta_s", c_double), ("T0", c_double),
                ("S0", c_double), ("f0", c_double), ("beta_plane", c_double),
                ("omega", c_double), ("radius", c_double), ("nu0", c_double),
                ("ri_a", c_double), ("nu_b", c_double), ("kappa_b", c_double),
                ("kappa_conv", c_double), ("weno_eps", c_double), ("weno_linear", c_int),
                ("min_depth", c_double), ("precision", c_int), ("closure", c_int),
                ("check_every", c_int), ("taux", POINTER(c_double)), ("tauy", POINTER(c_double)),
                ("closure_hidden", c_int), ("baro_filter", c_int), ("vertical_weno", c_int),
                ("momentum_vadv", c_int)]


class OceanBatch(ctypes.Structure):
    _fields_ = [(n, c_void_p) for n in ("X", "dzT", "dzS", "FT", "FS", "GT", "GS", "face", "wet")]


class ClosureScales(ctypes.Structure):
    _fields_ = [(n, ctypes.c_float) for n in ("kappa", "gT", "gS", "sFT", "sFS", "sGT", "sGS")]


class OceanDiag(ctypes.Structure):
    _fields_ = [("step", c_long), ("tracer_T", c_double), ("tracer_S", c_double),
                ("volume_eta", c_double), ("ke", c_double), ("max_cfl", c_double),
                ("wet_volume", c_double), ("nonfinite", c_int)]


_lib = None
_lock = threading.Lock()


class OceanError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{OCEAN_ERR.get(code, code)}: {msg}")
        self.code = code


def library_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True) -> ctypes.CDLL:
    """Load libocean.so (building it in-tree first when sources changed)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_needed and _build.needs_build():
            _build.build()
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libocean.so not built ({path}); run paper_2309_06662_gb300.build")
        L = ctypes.CDLL(path)
        pv, pd, pf = c_void_p, POINTER(c_double), POINTER(ctypes.c_float)
        sig = {
            "ocean_arena_bytes": (c_int, [POINTER(OceanGrid), POINTER(OceanParams), POINTER(c_size_t)]),
            "ocean_create": (c_int, [POINTER(OceanGrid), pd, POINTER(OceanParams), POINTER(pv)]),
            "ocean_create_in": (c_int, [POINTER(OceanGrid), pd, POINTER(OceanParams), pv, c_size_t,
                                        pv, POINTER(pv)]),
            "ocean_destroy": (None, [pv]),
            "ocean_last_error": (ctypes.c_char_p, [pv]),
            "ocean_set_field": (c_int, [pv, c_int, pd, c_size_t]),
            "ocean_get_field": (c_int, [pv, c_int, pd, c_size_t]),
            "ocean_set_wind_stress": (c_int, [pv, pd, pd]),
            "ocean_set_wind_stress_f32": (c_int, [pv, pf, pf]),
            "ocean_get_reference": (c_int, [pv, pd, pd]),
            "ocean_set_reference": (c_int, [pv, pd, pd]),
            "ocean_step": (c_int, [pv, c_int]),
            "ocean_step_async": (c_int, [pv, c_int]),
            "ocean_sync": (c_int, [pv]),
            "ocean_tendencies": (c_int, [pv]),
            "ocean_diagnostics": (c_int, [pv, POINTER(OceanDiag)]),
            "ocean_get_step": (c_long, [pv]),
            "ocean_set_step": (c_int, [pv, c_long]),
            "ocean_stream": (pv, [pv]),
            "ocean_profile": (c_int, [pv, c_int]),
            "ocean_phase_times": (c_int, [pv, pd, c_int, POINTER(c_long)]),
            "ocean_kernel_launches": (c_long, [pv]),
            "ocean_weno_faces": (c_int, [pv, pv, pv, c_int, pv, c_int, c_double, c_int, pv]),
            "ocean_tridiag_batched": (c_int, [pv, pv, pv, pv, pv, c_int, c_int, c_int, pv]),
            "ocean_tridiag_batched_static": (c_int, [pv, pv, pv, pv, pv, c_int, c_int, c_int, pv]),
            "ocean_mlp_param_count": (c_size_t, [c_int, c_int]),
            "ocean_set_closure": (c_int, [pv, POINTER(ctypes.c_float), c_size_t, POINTER(ctypes.c_float),
                                          POINTER(ctypes.c_float), POINTER(ClosureScales)]),
            "ocean_closure_features": (c_int, [pv, POINTER(ctypes.c_float), POINTER(ctypes.c_float),
                                               pv, pv, pv, pv, pv]),
            "ocean_coarse_grain": (c_int, [pv, pv, c_int, pv, pv, pv, pv]),
            "ocean_closure_targets": (c_int, [pv, pv, pv, pv, pv, pv, pv]),
            "ocean_mlp_create": (c_int, [c_int, c_int, c_int, POINTER(ctypes.c_float), pv, POINTER(pv)]),
            "ocean_mlp_destroy": (None, [pv]),
            "ocean_mlp_set_params": (c_int, [pv, POINTER(ctypes.c_float), c_size_t]),
            "ocean_mlp_get_params": (c_int, [pv, POINTER(ctypes.c_float), c_size_t]),
            "ocean_mlp_forward": (c_int, [pv, pv, c_int, pv]),
            "ocean_mlp_forward_bf16": (c_int, [pv, pv, c_int, pv]),
            "ocean_selftest_bounded_wait": (c_int, [ctypes.c_longlong, pv]),
            "ocean_mlp_loss_grad": (c_int, [pv, POINTER(OceanBatch), c_int, POINTER(ClosureScales),
                                            POINTER(ctypes.c_float), POINTER(ctypes.c_float)]),
            "ocean_mlp_train_step": (c_int, [pv, POINTER(OceanBatch), c_int, POINTER(ClosureScales),
                                             ctypes.c_float, POINTER(ctypes.c_float)]),
            "ocean_ensemble_create": (c_int, [c_int, POINTER(OceanGrid), POINTER(pd),
                                              POINTER(OceanParams), POINTER(pv)]),
            "ocean_ensemble_destroy": (None, [pv]),
            "ocean_ensemble_size": (c_int, [pv]),
            "ocean_ensemble_member": (pv, [pv, c_int]),
            "ocean_ensemble_stream": (pv, [pv]),
            "ocean_ensemble_step": (c_int, [pv, c_int]),
            "ocean_ensemble_step_async": (c_int, [pv, c_int]),
            "ocean_ensemble_autotune": (c_int, [pv, c_int, POINTER(c_int)]),
            "ocean_ensemble_autotune_regions": (c_int, [pv, c_int, POINTER(c_int)]),
            "ocean_ensemble_region_substeps": (c_int, [pv]),
            "ocean_ensemble_set_region_substeps": (c_int, [pv, c_int]),
            "ocean_ensemble_region_times": (c_int, [pv, POINTER(ctypes.c_float)]),
            "ocean_ensemble_launch_shapes": (c_int, [pv, POINTER(c_int), POINTER(c_int), POINTER(c_int)]),
            "ocean_ensemble_kernel_launches": (c_long, [pv]),
            "ocean_ensemble_kind_times": (c_int, [pv, pd]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
        return L


def header_functions(path: str = HEADER):
    """Names of the functions include/ocean.h declares."""
    txt = open(path).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(ocean_[a-z0-9_]+)\s*\(", txt)))


def _check(rc: int, h=None) -> None:
    if rc != OCEAN_OK:
        msg = load().ocean_last_error(h)
        raise OceanError(rc, msg.decode() if msg else "")


def _dp(a: np.ndarray):
    return a.ctypes.data_as(POINTER(c_double))


def _torch_cuda():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("libocean needs a CUDA device; none is visible")
    return torch


def make_grid(case):
    zf = np.ascontiguousarray(case.z_faces, dtype=np.float64)
    g = OceanGrid(case.kind, case.nx, case.ny, case.nz, int(case.periodic_x),
                  int(case.periodic_y), case.x0, case.x1, case.y0, case.y1, _dp(zf))
    return g, zf


def make_params(p: Dict[str, float], precision: int, taux=None, tauy=None, closure: int = 0,
                check_every: int = 0, closure_hidden: int = 0):
    keep = []
    tx = ty = None
    if taux is not None:
        tx = np.ascontiguousarray(taux, dtype=np.float64)
        keep.append(tx)
    if tauy is not None:
        ty = np.ascontiguousarray(tauy, dtype=np.float64)
        keep.append(ty)
    prm = OceanParams(
        p["dt"], int(p["n_substeps"]), p["chi"], p["g"], p["rho0"], p["alpha"], p["beta_s"],
        p["T0"], p["S0"], p["f0"], p["beta_plane"], p["omega"], p["radius"], p["nu0"], p["ri_a"],
        p["nu_b"], p["kappa_b"], p["kappa_conv"], p["weno_eps"], int(p["weno_linear"]),
        p["min_depth"], precision, closure, check_every,
        _dp(tx) if tx is not None else None, _dp(ty) if ty is not None else None,
        closure_hidden, int(p.get("baro_filter", 0)), int(p.get("vertical_weno", 0)),
        int(p.get("momentum_vadv", 0)))
    return prm, keep


class Ocean:
    """One model handle on the current CUDA device, in a torch-allocated arena."""

    def __init__(self, case, precision: int = OCEAN_FP64, params: Optional[dict] = None,
                 check_every: int = 0, own_memory: bool = False, closure: int = OCEAN_CLOSURE_RI,
                 closure_hidden: int = 0):
        torch = _torch_cuda()
        L = load()
        p = dict(case.params)
        if params:
            p.update(params)
        self.params = p
        self.nx, self.ny, self.nz = case.nx, case.ny, case.nz
        self.precision = precision
        grid, self._zf = make_grid(case)
        prm, self._keep = make_params(p, precision, case.taux, case.tauy, closure=closure,
                                      check_every=check_every, closure_hidden=closure_hidden)
        depth = np.ascontiguousarray(case.depth, dtype=np.float64)
        h = c_void_p()
        self._arena = None
        if own_memory:
            _check(L.ocean_create(ctypes.byref(grid), _dp(depth), ctypes.byref(prm), ctypes.byref(h)))
        else:
            nbytes = c_size_t()
            _check(L.ocean_arena_bytes(ctypes.byref(grid), ctypes.byref(prm), ctypes.byref(nbytes)))
            self._arena = torch.empty(nbytes.value + 256, dtype=torch.uint8, device="cuda")
            base = self._arena.data_ptr()
            aligned = (base + 255) & ~255
            stream = torch.cuda.current_stream().cuda_stream
            _check(L.ocean_create_in(ctypes.byref(grid), _dp(depth), ctypes.byref(prm),
                                     c_void_p(aligned), nbytes.value, c_void_p(stream),
                                     ctypes.byref(h)))
        self._h = h
        self.set("T", case.T)
        self.set("S", case.S)
        if case.u is not None:
            self.set("u", case.u)
        if case.v is not None:
            self.set("v", case.v)
        if case.eta is not None:
            self.set("eta", case.eta)

    @classmethod
    def _member(cls, handle, case, precision: int, params: dict):
        """A handle owned by an Ensemble (never destroyed here), set to the case's state."""
        self = cls.__new__(cls)
        self.params = params
        self.nx, self.ny, self.nz = case.nx, case.ny, case.nz
        self.precision = precision
        self._arena = None
        self._borrowed = True
        self._h = c_void_p(handle)
        self.set("T", case.T)
        self.set("S", case.S)
        if case.u is not None:
            self.set("u", case.u)
        if case.v is not None:
            self.set("v", case.v)
        if case.eta is not None:
            self.set("eta", case.eta)
        return self

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and not getattr(self, "_borrowed", False):
            load().ocean_destroy(h)
        self._h = None
        self._arena = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def shape(self, name: str):
        """Shape of field `name` as it crosses the ABI: (nz, ny, nx) or (ny, nx)."""
        return (self.ny, self.nx) if name in FIELDS_2D else (self.nz, self.ny, self.nx)

    def set(self, name: str, arr) -> None:
        """Copy a host field in (ocean_set_field; FP64, [k][j][i], k = 0 bottom)."""
        a = np.ascontiguousarray(arr, dtype=np.float64)
        assert a.shape == self.shape(name), (name, a.shape)
        _check(load().ocean_set_field(self._h, FIELD[name], _dp(a), a.size), self._h)

    def get(self, name: str) -> np.ndarray:
        """Copy a field out (ocean_get_field) as a new FP64 array."""
        out = np.zeros(self.shape(name))
        _check(load().ocean_get_field(self._h, FIELD[name], _dp(out), out.size), self._h)
        return out

    def step(self, n: int = 1) -> None:
        """Advance n steps and wait for them (ocean_step, with the health check)."""
        _check(load().ocean_step(self._h, int(n)), self._h)

    def step_async(self, n: int = 1) -> None:
        """Enqueue n steps on the model's stream without waiting (ocean_step_async)."""
        _check(load().ocean_step_async(self._h, int(n)), self._h)

    def sync(self) -> None:
        """Wait for the model's stream; device waits that gave up raise OceanError."""
        _check(load().ocean_sync(self._h), self._h)

    def tendencies(self) -> None:
        """Diagnostics and tendencies G^n of the current state without stepping."""
        _check(load().ocean_tendencies(self._h), self._h)

    def get_reference(self):
        T = np.zeros(self.nz)
        S = np.zeros(self.nz)
        _check(load().ocean_get_reference(self._h, _dp(T), _dp(S)), self._h)
        return T, S

    def set_reference(self, Tref, Sref) -> None:
        T = np.ascontiguousarray(Tref, dtype=np.float64)
        S = np.ascontiguousarray(Sref, dtype=np.float64)
        assert T.shape == (self.nz,) and S.shape == (self.nz,)
        _check(load().ocean_set_reference(self._h, _dp(T), _dp(S)), self._h)

    def checkpoint(self) -> Dict[str, np.ndarray]:
        """The complete restart state (host arrays)."""
        d = {f: self.get(f) for f in CHECKPOINT_FIELDS}
        d["Tref"], d["Sref"] = self.get_reference()
        d["step"] = np.array(self.nstep)
        return d

    def restore(self, d: Dict[str, np.ndarray]) -> None:
        """Resume from checkpoint(): the continuation is the same bit for bit."""
        self.set_reference(d["Tref"], d["Sref"])
        for f in CHECKPOINT_FIELDS:
            self.set(f, d[f])
        self.nstep = int(d["step"])

    # ---- learned closure
    def set_closure(self, params, mu, sigma, scales: dict) -> None:
        flat = flatten_params(params)
        m = np.ascontiguousarray(mu, dtype=np.float32)
        sg = np.ascontiguousarray(sigma, dtype=np.float32)
        sc = ClosureScales(**scales)
        _check(load().ocean_set_closure(self._h, _fp(flat), flat.size, _fp(m), _fp(sg),
                                        ctypes.byref(sc)), self._h)

    def closure_features(self, mu=None, sigma=None):
        """Device (torch) features X [ncol, 6nz] (with mu, sigma), masks and gradients."""
        torch = _torch_cuda()
        nc, nz = self.nx * self.ny, self.nz
        out = dict(face=torch.empty((nc, nz), dtype=torch.uint8, device="cuda"),
                   wet=torch.empty((nc, nz), dtype=torch.uint8, device="cuda"),
                   dzT=torch.empty((nc, nz), dtype=torch.float32, device="cuda"),
                   dzS=torch.empty((nc, nz), dtype=torch.float32, device="cuda"))
        Xp = None
        m = sg = None
        if mu is not None:
            out["X"] = torch.empty((nc, 6 * nz), dtype=torch.float32, device="cuda")
            Xp = c_void_p(out["X"].data_ptr())
            m = np.ascontiguousarray(mu, dtype=np.float32)
            sg = np.ascontiguousarray(sigma, dtype=np.float32)
        _check(load().ocean_closure_features(
            self._h, _fp(m) if m is not None else None, _fp(sg) if sg is not None else None, Xp,
            c_void_p(out["face"].data_ptr()), c_void_p(out["wet"].data_ptr()),
            c_void_p(out["dzT"].data_ptr()), c_void_p(out["dzS"].data_ptr())), self._h)
        return out

    def coarse_grain_to(self, coarse, r: int):
        """Coarse-grain this (fine) model onto `coarse`; returns the device targets."""
        torch = _torch_cuda()
        nc, nz = coarse.nx * coarse.ny, coarse.nz
        t = {k: torch.empty((nc, nz), dtype=torch.float32, device="cuda")
             for k in ("FT", "FS", "GTm", "GSm")}
        _check(load().ocean_coarse_grain(self._h, coarse._h, r,
                                         *(c_void_p(t[k].data_ptr()) for k in ("FT", "FS", "GTm", "GSm"))),
               self._h)
        return t

    def closure_targets(self, t):
        """Lateral residual targets (after tendencies()) into t["GT"], t["GS"]."""
        torch = _torch_cuda()
        nc, nz = self.nx * self.ny, self.nz
        t["GT"] = torch.empty((nc, nz), dtype=torch.float32, device="cuda")
        t["GS"] = torch.empty((nc, nz), dtype=torch.float32, device="cuda")
        _check(load().ocean_closure_targets(
            self._h, *(c_void_p(t[k].data_ptr()) for k in ("GTm", "GSm", "FT", "FS", "GT", "GS"))),
            self._h)
        return t

    def set_wind_stress(self, taux, tauy) -> None:
        """Replace the surface wind stress ([ny][nx], N/m^2); the arrays are copied.
        Two float32 arrays go through ocean_set_wind_stress_f32 (half the bytes), anything
        else as float64."""
        if getattr(taux, "dtype", None) == np.float32 and getattr(tauy, "dtype", None) == np.float32:
            tx, ty = np.ascontiguousarray(taux), np.ascontiguousarray(tauy)
            _check(load().ocean_set_wind_stress_f32(self._h, _fp(tx), _fp(ty)), self._h)
            return
        tx = np.ascontiguousarray(taux, dtype=np.float64)
        ty = np.ascontiguousarray(tauy, dtype=np.float64)
        _check(load().ocean_set_wind_stress(self._h, _dp(tx), _dp(ty)), self._h)

    def diagnostics(self) -> Dict[str, float]:
        """Conservation and health sums of the current state (ocean_diagnostics)."""
        d = OceanDiag()
        _check(load().ocean_diagnostics(self._h, ctypes.byref(d)), self._h)
        return dict(step=d.step, tracer_T=d.tracer_T, tracer_S=d.tracer_S,
                    volume_eta=d.volume_eta, ke=d.ke, max_cfl=d.max_cfl,
                    wet_volume=d.wet_volume, nonfinite=bool(d.nonfinite))

    @property
    def nstep(self) -> int:
        return load().ocean_get_step(self._h)

    @nstep.setter
    def nstep(self, n: int) -> None:
        _check(load().ocean_set_step(self._h, int(n)), self._h)

    PHASES = ["diag", "tracer", "momentum", "barotropic", "correct"]

    def profile(self, enable: bool) -> None:
        _check(load().ocean_profile(self._h, int(enable)), self._h)

    def phase_times(self):
        ms = np.zeros(len(self.PHASES))
        n = c_long()
        _check(load().ocean_phase_times(self._h, _dp(ms), len(ms), ctypes.byref(n)), self._h)
        return dict(zip(self.PHASES, ms.tolist())), n.value

    @property
    def launches(self) -> int:
        return load().ocean_kernel_launches(self._h)

    @property
    def stream(self) -> int:
        return load().ocean_stream(self._h) or 0


def weno_faces(q, vel, inside=None, precision: int = OCEAN_FP64, eps: float = 1e-30,
               linear: bool = False):
    """ocean_weno_faces on torch CUDA tensors (returns a new tensor)."""
    torch = _torch_cuda()
    dt = torch.float64 if precision == OCEAN_FP64 else torch.float32
    q = q.to(device="cuda", dtype=dt).contiguous()
    vel = vel.to(device="cuda", dtype=dt).contiguous()
    out = torch.empty_like(q)
    ins = None
    if inside is not None:
        ins = inside.to(device="cuda", dtype=torch.uint8).contiguous()
    s = torch.cuda.current_stream().cuda_stream
    rc = load().ocean_weno_faces(c_void_p(q.data_ptr()), c_void_p(vel.data_ptr()),
                                 c_void_p(ins.data_ptr()) if ins is not None else None,
                                 q.numel(), c_void_p(out.data_ptr()), precision, eps, int(linear),
                                 c_void_p(s))
    _check(rc)
    return out


def tridiag_batched(a, b, c, d, precision: int = OCEAN_FP64):
    """ocean_tridiag_batched on level-major [n, nsys] torch CUDA tensors."""
    torch = _torch_cuda()
    dt = torch.float64 if precision == OCEAN_FP64 else torch.float32
    a, b, c, d = (t.to(device="cuda", dtype=dt).contiguous() for t in (a, b, c, d))
    x = torch.empty_like(d)
    n, nsys = d.shape
    s = torch.cuda.current_stream().cuda_stream
    rc = load().ocean_tridiag_batched(*(c_void_p(t.data_ptr()) for t in (a, b, c, d)),
                                      c_void_p(x.data_ptr()), n, nsys, precision, c_void_p(s))
    _check(rc)
    return x


# ----------------------------------------------------------------------------- closure network

def flatten_params(params) -> np.ndarray:
    """[(W [in, out], b [out])...] -> the flat float32 layout of the C ABI."""
    return np.concatenate([np.concatenate([W.reshape(-1), b.reshape(-1)]) for W, b in params]
                          ).astype(np.float32)


def unflatten_params(flat: np.ndarray, dims):
    out, o = [], 0
    for a, b in zip(dims[:-1], dims[1:]):
        W = flat[o:o + a * b].reshape(a, b)
        o += a * b
        out.append((W, flat[o:o + b]))
        o += b
    return out


def _fp(a: np.ndarray):
    return a.ctypes.data_as(POINTER(ctypes.c_float))


class MLP:
    """The closure network's trainer handle (ocean_mlp_*) on torch's current stream."""

    def __init__(self, nz: int, hidden: int, max_batch: int, params=None):
        torch = _torch_cuda()
        L = load()
        self.nz, self.hidden, self.max_batch = nz, hidden, max_batch
        self.dims = [6 * nz, hidden, hidden, hidden, 3 * nz]
        self.count = L.ocean_mlp_param_count(nz, hidden)
        flat = flatten_params(params) if params is not None else None
        h = c_void_p()
        stream = torch.cuda.current_stream().cuda_stream
        _check(L.ocean_mlp_create(nz, hidden, max_batch, _fp(flat) if flat is not None else None,
                                  c_void_p(stream), ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().ocean_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self):
        flat = np.zeros(self.count, dtype=np.float32)
        _check(load().ocean_mlp_get_params(self._h, _fp(flat), flat.size))
        return unflatten_params(flat.astype(np.float64), self.dims)

    def set_params(self, params) -> None:
        flat = flatten_params(params)
        _check(load().ocean_mlp_set_params(self._h, _fp(flat), flat.size))

    def forward(self, X):
        """X: torch CUDA float32 [M, 6nz] -> Y [M, 3nz]."""
        torch = _torch_cuda()
        X = X.to(device="cuda", dtype=torch.float32).contiguous()
        Y = torch.empty((X.shape[0], self.dims[-1]), device="cuda", dtype=torch.float32)
        _check(load().ocean_mlp_forward(self._h, c_void_p(X.data_ptr()), X.shape[0],
                                        c_void_p(Y.data_ptr())))
        return Y

    def forward_bf16(self, Xb):
        """Xb: torch CUDA bfloat16 [M, 6nz] -> Y [M, 3nz] (no input conversion)."""
        torch = _torch_cuda()
        Xb = Xb.to(device="cuda", dtype=torch.bfloat16).contiguous()
        Y = torch.empty((Xb.shape[0], self.dims[-1]), device="cuda", dtype=torch.float32)
        _check(load().ocean_mlp_forward_bf16(self._h, c_void_p(Xb.data_ptr()), Xb.shape[0],
                                             c_void_p(Y.data_ptr())))
        return Y

    @staticmethod
    def batch(tensors):
        """ocean_batch from a dict of torch CUDA tensors (float32 / uint8, contiguous)."""
        b = OceanBatch()
        for k in ("X", "dzT", "dzS", "FT", "FS", "GT", "GS", "face", "wet"):
            setattr(b, k, tensors[k].data_ptr())
        return b

    def loss_grad(self, tensors, scales: dict, grads: bool = True):
        b = self.batch(tensors)
        sc = ClosureScales(**scales)
        loss = ctypes.c_float()
        g = np.zeros(self.count, dtype=np.float32) if grads else None
        _check(load().ocean_mlp_loss_grad(self._h, ctypes.byref(b), tensors["X"].shape[0],
                                          ctypes.byref(sc), ctypes.byref(loss),
                                          _fp(g) if g is not None else None))
        return loss.value, (unflatten_params(g.astype(np.float64), self.dims) if grads else None)

    def train_step(self, tensors, scales: dict, lr: float) -> float:
        b = self.batch(tensors)
        sc = ClosureScales(**scales)
        loss = ctypes.c_float()
        _check(load().ocean_mlp_train_step(self._h, ctypes.byref(b), tensors["X"].shape[0],
                                           ctypes.byref(sc), lr, ctypes.byref(loss)))
        return loss.value


# ----------------------------------------------------------------------------- ensemble

ENS_KINDS = ["diag", "tracer", "momentum", "baro_begin", "baro_pass", "baro_end", "correct"]


class Ensemble:
    """ocean_ensemble_*: many closed-basin models stepped together by persistent kernels
    over a (member, tile) work list, one CUDA graph per step."""

    def __init__(self, cases, precision: int = OCEAN_MIXED, params: Optional[dict] = None):
        _torch_cuda()
        L = load()
        M = len(cases)
        grids = (OceanGrid * M)()
        prms = (OceanParams * M)()
        depths = (POINTER(c_double) * M)()
        self._keep = []
        plist = []
        for i, c in enumerate(cases):
            p = dict(c.params)
            if params:
                p.update(params)
            plist.append(p)
            g, zf = make_grid(c)
            pr, keep = make_params(p, precision, c.taux, c.tauy)
            d = np.ascontiguousarray(c.depth, dtype=np.float64)
            self._keep += [zf, keep, d]
            grids[i] = g
            prms[i] = pr
            depths[i] = _dp(d)
        h = c_void_p()
        _check(L.ocean_ensemble_create(M, grids, depths, prms, ctypes.byref(h)))
        self._h = h
        self.precision = precision
        self.members = [Ocean._member(L.ocean_ensemble_member(h, i), c, precision, plist[i])
                        for i, c in enumerate(cases)]
        self.cells = int(sum(c.nx * c.ny * c.nz for c in cases))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            for m in self.members:
                m._h = None
            load().ocean_ensemble_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __len__(self):
        return len(self.members)

    def step(self, n: int = 1) -> None:
        _check(load().ocean_ensemble_step(self._h, int(n)))

    def step_async(self, n: int = 1) -> None:
        _check(load().ocean_ensemble_step_async(self._h, int(n)))

    def sync(self) -> None:
        self.members[0].sync()

    def autotune(self, reps: int = 1) -> int:
        """Tune the launch shapes on real steps; returns the number of steps taken."""
        n = c_int()
        _check(load().ocean_ensemble_autotune(self._h, int(reps), ctypes.byref(n)))
        return n.value

    def autotune_regions(self, reps: int = 1) -> int:
        """Tune the barotropic region's halo width (substeps per pass: 4, 6 or 8) on real
        steps; returns the number of steps taken."""
        n = c_int()
        _check(load().ocean_ensemble_autotune_regions(self._h, int(reps), ctypes.byref(n)))
        return n.value

    @property
    def region_substeps(self) -> int:
        return load().ocean_ensemble_region_substeps(self._h)

    @region_substeps.setter
    def region_substeps(self, bs: int) -> None:
        _check(load().ocean_ensemble_set_region_substeps(self._h, int(bs)))

    def region_times(self):
        """Sub-cycle ms per step measured by autotune_regions for halo widths 4, 6, 8."""
        ms = (ctypes.c_float * 3)()
        _check(load().ocean_ensemble_region_times(self._h, ms))
        return dict(zip((4, 6, 8), [float(x) for x in ms]))

    def launch_shapes(self):
        g, d, w = ((c_int * len(ENS_KINDS))() for _ in range(3))
        _check(load().ocean_ensemble_launch_shapes(self._h, g, d, w))
        return {k: dict(grid=g[i], dynamic=bool(d[i]), items=w[i]) for i, k in enumerate(ENS_KINDS)}

    def kind_times(self):
        """Device ms per step of each kernel kind under its tuned shape (after autotune)."""
        ms = np.zeros(len(ENS_KINDS))
        _check(load().ocean_ensemble_kind_times(self._h, _dp(ms)))
        return dict(zip(ENS_KINDS, ms.tolist()))

    @property
    def launches(self) -> int:
        return load().ocean_ensemble_kernel_launches(self._h)

    @property
    def stream(self) -> int:
        return load().ocean_ensemble_stream(self._h) or 0
