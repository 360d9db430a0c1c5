"""Plain FP64 oracle of the learned column closure (test infrastructure only).

A column MLP stands in for the subgrid vertical and lateral tracer-flux
parameterisation.  The paper itself uses a Richardson-number closure (Sec. "How
performance was measured"); the learned closure, its inputs, targets and loss are the
design this repository implements, written here in plain numpy so the CUDA kernels can
be checked against it:

  features   per wet column: T, S, centre-averaged u, v at the nz levels, N^2 and S^2
             (shear squared) on the nz bottom faces (0 on the sea-floor face), z-scored
             with per-feature statistics; 0 on dry levels;
  network    6 nz -> H -> H -> H -> 3 nz, SiLU after each hidden layer;
  outputs    kappa_k = kappa_scale softplus(y_k) on interior wet faces, added to the
             Richardson-number diffusivity (the network supplies the resolved-eddy
             flux that the coarse grid misses; convective and background mixing stay
             with the Richardson-number closure, as in the fine run), and tracer
             tendency corrections dG_T = gT_scale y_{nz+k}, dG_S = gS_scale y_{2nz+k};
  loss       mean squared error of the parameterised vertical flux -kappa dz<T> (and
             S) against the coarse-grained subgrid flux <wT> - <w><T>, plus that of dG
             against the lateral residual, each normalised by its target scale;
  optimiser  Adam (Kingma & Ba 2015);
  targets    4 x 4 coarse-graining of a fine run of the same solver.
"""
from __future__ import annotations

import math
from typing import Dict, List, Tuple

import numpy as np


# ----------------------------------------------------------------------------- bf16

def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    u = (u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


# ----------------------------------------------------------------------------- features

def column_features(T, S, u, v, kb, zf, g, alpha, beta_s, periodic_x: bool, periodic_y: bool):
    """Raw features [ny*nx, 6 nz] and their wet mask from full 3-D fields [nz, ny, nx].

    u, v are face values (west, south faces; 0 on dry faces); kb is the lowest wet level
    of each column (nz for land).  Order: T, S, ubar, vbar, N^2, Sh^2.
    """
    nz, ny, nx = T.shape
    zc = 0.5 * (zf[1:] + zf[:-1])
    dzf = np.zeros(nz)
    dzf[1:] = zc[1:] - zc[:-1]
    uE = np.roll(u, -1, axis=2) if periodic_x else np.concatenate([u[:, :, 1:], np.zeros((nz, ny, 1))], axis=2)
    vN = np.roll(v, -1, axis=1) if periodic_y else np.concatenate([v[:, 1:, :], np.zeros((nz, 1, nx))], axis=1)
    ub = 0.5 * (u + uE)
    vb = 0.5 * (v + vN)
    k = np.arange(nz)[:, None, None]
    wet = k >= kb[None, :, :]
    face = k >= kb[None, :, :] + 1          # interior faces (bottom face of level k > kb)
    n2 = np.zeros_like(T)
    sh2 = np.zeros_like(T)
    dT = T[1:] - T[:-1]
    dS = S[1:] - S[:-1]
    n2[1:] = g * (alpha * dT - beta_s * dS) / dzf[1:, None, None]
    sh2[1:] = ((ub[1:] - ub[:-1]) ** 2 + (vb[1:] - vb[:-1]) ** 2) / (dzf[1:, None, None] ** 2)
    n2 = np.where(face, n2, 0.0)
    sh2 = np.where(face, sh2, 0.0)
    blocks = [np.where(wet, T, 0.0), np.where(wet, S, 0.0), np.where(wet, ub, 0.0),
              np.where(wet, vb, 0.0), n2, sh2]
    masks = [wet, wet, wet, wet, face, face]
    raw = np.concatenate([b.reshape(nz, -1).T for b in blocks], axis=1)
    msk = np.concatenate([m.reshape(nz, -1).T for m in masks], axis=1)
    return raw, msk


def normalise(raw: np.ndarray, msk: np.ndarray, mu: np.ndarray, sigma: np.ndarray) -> np.ndarray:
    """z-score each feature on its wet entries; 0 elsewhere."""
    return np.where(msk, (raw - mu[None, :]) / sigma[None, :], 0.0)


# ----------------------------------------------------------------------------- MLP

def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def softplus(z):
    return np.where(z > 20.0, z, np.log1p(np.exp(np.minimum(z, 20.0))))


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def mlp_forward(params: List[Tuple[np.ndarray, np.ndarray]], X: np.ndarray, bf16: bool = False):
    """Y = MLP(X); params = [(W [in, out], b [out])...]; with bf16, the operands of every
    GEMM (inputs, weights, hidden activations) are rounded to bfloat16 first, as on the
    tensor cores.  Returns (Y, cache)."""
    rnd = bf16_round if bf16 else (lambda a: a)
    a = rnd(X)
    cache = []
    for li, (W, b) in enumerate(params):
        z = a @ rnd(W) + b
        cache.append((a, z))
        if li < len(params) - 1:
            a = rnd(silu(z))
        else:
            a = z
    return a, cache


def mlp_backward(params, cache, dY, bf16: bool = False):
    """Gradients [(dW, db)...] of sum(dY * Y) with respect to the parameters."""
    rnd = bf16_round if bf16 else (lambda x: x)
    grads = [None] * len(params)
    d = dY
    for li in range(len(params) - 1, -1, -1):
        W, _ = params[li]
        a, z = cache[li]
        if li < len(params) - 1:
            d = d * silu_grad(z)
        grads[li] = (a.T @ d, d.sum(axis=0))
        if li > 0:
            d = d @ rnd(W).T
    return grads


# ----------------------------------------------------------------------------- closure head

def closure_outputs(Y: np.ndarray, nz: int, scales: Dict[str, float]):
    """kappa (softplus, scaled), dG_T, dG_S from the network outputs [ncol, 3 nz]."""
    kap = scales["kappa"] * softplus(Y[:, :nz])
    dgt = scales["gT"] * Y[:, nz:2 * nz]
    dgs = scales["gS"] * Y[:, 2 * nz:]
    return kap, dgt, dgs


def closure_loss(Y, nz, scales, dzT, dzS, FT, FS, GT, GS, face, wet):
    """Normalised loss and its gradient with respect to Y.

    dzT, dzS, FT, FS on faces [ncol, nz] (face mask `face`); GT, GS targets on levels
    (mask `wet`).  L = mean_face[((-kap dzT - FT)/sFT)^2 + ((-kap dzS - FS)/sFS)^2]
                     + mean_wet[((dGT - GT)/sGT)^2 + ((dGS - GS)/sGS)^2].
    """
    kap, dgt, dgs = closure_outputs(Y, nz, scales)
    nf = max(1, int(face.sum()))
    nw = max(1, int(wet.sum()))
    rT = np.where(face, (-kap * dzT - FT) / scales["sFT"], 0.0)
    rS = np.where(face, (-kap * dzS - FS) / scales["sFS"], 0.0)
    qT = np.where(wet, (dgt - GT) / scales["sGT"], 0.0)
    qS = np.where(wet, (dgs - GS) / scales["sGS"], 0.0)
    L = (np.sum(rT ** 2) + np.sum(rS ** 2)) / nf + (np.sum(qT ** 2) + np.sum(qS ** 2)) / nw
    dkap = (2.0 * rT * (-dzT) / scales["sFT"] + 2.0 * rS * (-dzS) / scales["sFS"]) / nf
    dY = np.zeros_like(Y)
    dY[:, :nz] = dkap * scales["kappa"] * sigmoid(Y[:, :nz])
    dY[:, nz:2 * nz] = 2.0 * qT / scales["sGT"] * scales["gT"] / nw
    dY[:, 2 * nz:] = 2.0 * qS / scales["sGS"] * scales["gS"] / nw
    return L, dY


# ----------------------------------------------------------------------------- Adam

def adam_step(w, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (in place on w, m, v); t is the 1-based step count."""
    m *= b1
    m += (1.0 - b1) * g
    v *= b2
    v += (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    w -= lr * mh / (np.sqrt(vh) + eps)


# ----------------------------------------------------------------------------- coarse-graining

def coarse_grain_mean(F: np.ndarray, wgt: np.ndarray, r: int) -> Tuple[np.ndarray, np.ndarray]:
    """Weighted r x r block means of F [..., ny, nx] with weights wgt (0 = excluded);
    returns (mean, summed weight), mean 0 where no weight."""
    *lead, ny, nx = F.shape
    Fw = (F * wgt).reshape(*lead, ny // r, r, nx // r, r).sum(axis=(-3, -1))
    W = np.broadcast_to(wgt, F.shape).reshape(*lead, ny // r, r, nx // r, r).sum(axis=(-3, -1))
    mean = np.where(W > 0, Fw / np.where(W > 0, W, 1.0), 0.0)
    return mean, W


def subgrid_vertical_flux(w, T, kb, area, r: int):
    """<w T_f> - <w><T_f> on the bottom faces, averaged over the wet fine faces of each
    r x r block (weights: fine cell areas); T_f = (T_k + T_{k-1})/2.  Face k = 0 is 0."""
    nz = T.shape[0]
    k = np.arange(nz)[:, None, None]
    face = (k >= kb[None] + 1).astype(float) * area[None, :, :]
    Tf = np.zeros_like(T)
    Tf[1:] = 0.5 * (T[1:] + T[:-1])
    wT, _ = coarse_grain_mean(w * Tf, face, r)
    wm, _ = coarse_grain_mean(w, face, r)
    Tm, _ = coarse_grain_mean(Tf, face, r)
    F = wT - wm * Tm
    F[0] = 0.0
    return F


# ----------------------------------------------------------------------------- in the model

def learned_fields(model, params, mu, sigma, scales, bf16: bool = True):
    """The learned closure's extra diffusivity (on interior wet faces) and tracer
    corrections (on wet cells) for an oracle model's current state, [nz, ny, nx] each; a
    column with any non-finite output gets neither (0)."""
    c = model.case
    p = model.params
    kb = model.kb_array()
    raw, msk = column_features(model.get("T"), model.get("S"), model.get("u"), model.get("v"),
                               kb, np.asarray(c.z_faces), p["g"], p["alpha"], p["beta_s"],
                               bool(c.periodic_x), bool(c.periodic_y))
    X = normalise(raw, msk, np.asarray(mu, float), np.asarray(sigma, float))
    Y, _ = mlp_forward(params, X, bf16=bf16)
    nz, ny, nx = model.nz, model.ny, model.nx
    kap, dgt, dgs = closure_outputs(Y, nz, scales)
    ok = np.all(np.isfinite(Y), axis=1)[:, None]
    k = np.arange(nz)[None, :]
    kbf = kb.reshape(-1)[:, None]
    face = (k >= kbf + 1) & ok
    wet = (k >= kbf) & ok
    K = np.where(face, kap, 0.0)
    A = np.where(wet, dgt, 0.0)
    B = np.where(wet, dgs, 0.0)
    shape = lambda Z: Z.T.reshape(nz, ny, nx)
    return shape(K), shape(A), shape(B)


def step_learned(model, nsteps, params, mu, sigma, scales, bf16: bool = True):
    """Advance an oracle model with the learned closure: before each step the network is
    evaluated on the current state and its diffusivity, added to the Richardson-number
    one of that state, and its corrections handed to the FP64 step."""
    for _ in range(nsteps):
        kap, dgt, dgs = learned_fields(model, params, mu, sigma, scales, bf16)
        model.tendencies()
        kri = model.get("kappa")
        model.set_closure_fields(kri + kap, dgt, dgs)
        model.step(1)
        model.set_closure_fields(None, None, None)


def coarse_grain_state(fine: dict, kbf, kbc, area_rows, r: int):
    """4-way coarse-graining of a fine state (the same operator as the CUDA path):
    fine = dict(u, v, T, S, w, GT, GS [nz, ny, nx], eta [ny, nx]); kbf / kbc the lowest
    wet levels of fine / coarse columns (kbu, kbv derived, periodic in x); area_rows the
    fine cell area per row.  Returns the coarse (u, v, T, S, eta) and FT, FS, GTm, GSm."""
    T = fine["T"]
    nz, ny, nx = T.shape
    Ny, Nx = ny // r, nx // r
    k = np.arange(nz)[:, None, None]
    area = np.broadcast_to(area_rows[:, None], (ny, nx))
    wetf = (k >= kbf[None]).astype(float) * area[None]
    out = {}
    for name in ("T", "S", "GT", "GS"):
        mean, _ = coarse_grain_mean(fine[name], wetf, r)
        out[name] = mean
    wetc = k >= kbc[None]
    for name in ("T", "S"):
        out[name] = np.where(wetc, out[name], 0.0)
    GTm = np.where(wetc, out.pop("GT"), 0.0)
    GSm = np.where(wetc, out.pop("GS"), 0.0)
    FT = subgrid_vertical_flux(fine["w"], fine["T"], kbf, area, r)
    FS = subgrid_vertical_flux(fine["w"], fine["S"], kbf, area, r)
    facec = k >= kbc[None] + 1
    FT = np.where(facec, FT, 0.0)
    FS = np.where(facec, FS, 0.0)
    # u on the coarse west faces: fine faces (r I, r J + b); v on south faces (r I + a, r J)
    kbuf = np.maximum(kbf, np.roll(kbf, 1, axis=1))
    kbvf = np.maximum(kbf, np.vstack([np.full((1, nx), nz), kbf[:-1]]))
    kbuc = np.maximum(kbc, np.roll(kbc, 1, axis=1))
    kbvc = np.maximum(kbc, np.vstack([np.full((1, Nx), nz), kbc[:-1]]))
    uw = (k >= kbuf[None]).astype(float)
    us = (fine["u"] * uw)[:, :, ::r].reshape(nz, Ny, r, Nx).sum(axis=2)
    un = uw[:, :, ::r].reshape(nz, Ny, r, Nx).sum(axis=2)
    out["u"] = np.where((k >= kbuc[None]) & (un > 0), us / np.maximum(un, 1), 0.0)
    vw = (k >= kbvf[None]).astype(float)
    vs = (fine["v"] * vw)[:, ::r, :].reshape(nz, Ny, Nx, r).sum(axis=3)
    vn = vw[:, ::r, :].reshape(nz, Ny, Nx, r).sum(axis=3)
    out["v"] = np.where((k >= kbvc[None]) & (vn > 0), vs / np.maximum(vn, 1), 0.0)
    colw = (kbf < nz).astype(float) * area
    eta, W = coarse_grain_mean(fine["eta"], colw, r)
    out["eta"] = np.where((kbc < nz) & (W > 0), eta, 0.0)
    return out, FT, FS, GTm, GSm
