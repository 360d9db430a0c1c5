"""Pins of the learned-closure oracle (CPU): gradients against central finite
differences and against torch autograd, bfloat16 rounding against torch's conversion,
Adam's first step in closed form, exact feature and coarse-graining invariants."""
import math

import numpy as np
import pytest

from oracle import closure as C
from paper_2309_06662_gb300 import inputs

NZ = 4
SCALES = dict(kappa=1e-2, gT=1e-6, gS=1e-7, sFT=1e-5, sFS=1e-6, sGT=1e-6, sGS=1e-7)


def _problem(seed=0, ncol=7, hidden=6):
    rng = np.random.default_rng(seed)
    dims = [6 * NZ, hidden, hidden, hidden, 3 * NZ]
    params = [(rng.normal(0, 0.5, (a, b)), rng.normal(0, 0.1, b)) for a, b in zip(dims[:-1], dims[1:])]
    X = rng.normal(size=(ncol, 6 * NZ))
    face = rng.random((ncol, NZ)) > 0.2
    wet = rng.random((ncol, NZ)) > 0.1
    tgt = dict(dzT=rng.normal(0, 1e-3, (ncol, NZ)), dzS=rng.normal(0, 1e-4, (ncol, NZ)),
               FT=rng.normal(0, 1e-5, (ncol, NZ)), FS=rng.normal(0, 1e-6, (ncol, NZ)),
               GT=rng.normal(0, 1e-6, (ncol, NZ)), GS=rng.normal(0, 1e-7, (ncol, NZ)))
    return params, X, face, wet, tgt


def _loss(params, X, face, wet, tgt):
    Y, cache = C.mlp_forward(params, X)
    L, dY = C.closure_loss(Y, NZ, SCALES, tgt["dzT"], tgt["dzS"], tgt["FT"], tgt["FS"],
                           tgt["GT"], tgt["GS"], face, wet)
    return L, dY, cache


def test_backprop_matches_central_differences():
    params, X, face, wet, tgt = _problem()
    L, dY, cache = _loss(params, X, face, wet, tgt)
    grads = C.mlp_backward(params, cache, dY)
    h = 1e-6
    rng = np.random.default_rng(1)
    for li, (W, b) in enumerate(params):
        for (arr, g) in ((W, grads[li][0]), (b, grads[li][1])):
            for _ in range(6):
                idx = tuple(rng.integers(0, s) for s in arr.shape)
                old = arr[idx]
                arr[idx] = old + h
                Lp = _loss(params, X, face, wet, tgt)[0]
                arr[idx] = old - h
                Lm = _loss(params, X, face, wet, tgt)[0]
                arr[idx] = old
                fd = (Lp - Lm) / (2 * h)
                assert abs(fd - g[idx]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (li, idx, fd, g[idx])


def test_backprop_matches_torch_autograd():
    torch = pytest.importorskip("torch")
    params, X, face, wet, tgt = _problem(seed=3, ncol=11, hidden=9)
    L, dY, cache = _loss(params, X, face, wet, tgt)
    grads = C.mlp_backward(params, cache, dY)
    tp = [(torch.tensor(W, requires_grad=True), torch.tensor(b, requires_grad=True)) for W, b in params]
    a = torch.tensor(X)
    for li, (W, b) in enumerate(tp):
        a = a @ W + b
        if li < len(tp) - 1:
            a = torch.nn.functional.silu(a)
    Y = a
    t = {k: torch.tensor(v) for k, v in tgt.items()}
    fm, wm = torch.tensor(face), torch.tensor(wet)
    kap = SCALES["kappa"] * torch.nn.functional.softplus(Y[:, :NZ])
    rT = torch.where(fm, (-kap * t["dzT"] - t["FT"]) / SCALES["sFT"], torch.zeros(()))
    rS = torch.where(fm, (-kap * t["dzS"] - t["FS"]) / SCALES["sFS"], torch.zeros(()))
    qT = torch.where(wm, (SCALES["gT"] * Y[:, NZ:2 * NZ] - t["GT"]) / SCALES["sGT"], torch.zeros(()))
    qS = torch.where(wm, (SCALES["gS"] * Y[:, 2 * NZ:] - t["GS"]) / SCALES["sGS"], torch.zeros(()))
    Lt = (rT.pow(2).sum() + rS.pow(2).sum()) / fm.sum() + (qT.pow(2).sum() + qS.pow(2).sum()) / wm.sum()
    Lt.backward()
    assert abs(Lt.item() - L) <= 1e-12 * abs(L)
    for (W, b), (gW, gb) in zip(tp, grads):
        np.testing.assert_allclose(gW, W.grad.numpy(), rtol=1e-10, atol=1e-14)
        np.testing.assert_allclose(gb, b.grad.numpy(), rtol=1e-10, atol=1e-14)


def test_bf16_round_matches_torch_conversion():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2)
    x = np.concatenate([rng.normal(size=1000) * 10.0 ** rng.integers(-8, 8, 1000),
                        [1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -2.5, 0.0, 65504.0]])
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(C.bf16_round(x), ref)


def test_adam_first_step_closed_form():
    # after one step m_hat = g and v_hat = g^2, so w moves by lr g / (|g| + eps)
    g = np.array([3.0, -0.5, 1e-3, 0.0])
    w = np.zeros(4)
    m = np.zeros(4)
    v = np.zeros(4)
    C.adam_step(w, g, m, v, 1, lr=0.01, eps=1e-8)
    np.testing.assert_allclose(w, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_features_linear_profiles():
    nz, ny, nx = 5, 3, 4
    zf = inputs.uniform_z_faces(nz, 1000.0)
    zc = 0.5 * (zf[1:] + zf[:-1])
    T = (10 + 0.01 * zc)[:, None, None] + np.zeros((nz, ny, nx))
    S = np.full((nz, ny, nx), 35.0)
    u = (0.1 + 1e-4 * zc)[:, None, None] + np.zeros((nz, ny, nx))
    v = np.zeros((nz, ny, nx))
    kb = np.zeros((ny, nx), dtype=int)
    kb[0, 0] = 2
    raw, msk = C.column_features(T, S, u, v, kb, zf, 9.80665, 2e-4, 8e-4, True, True)
    n2 = raw[:, 4 * nz:5 * nz]
    sh2 = raw[:, 5 * nz:]
    # N^2 = g alpha dT/dz and S^2 = (du/dz)^2 on interior faces; 0 on the sea-floor face
    assert np.allclose(n2[1:, 1:], 9.80665 * 2e-4 * 0.01, rtol=1e-12)
    assert np.allclose(sh2[1:, 1:], 1e-8, rtol=1e-9)
    assert np.all(n2[:, 0] == 0.0)
    assert np.all(n2[0, :3] == 0.0) and np.all(~msk[0, 4 * nz:4 * nz + 3])
    assert np.all(raw[0, :2] == 0.0)            # dry levels of the shallow column


def test_coarse_graining_invariants():
    rng = np.random.default_rng(4)
    nz, ny, nx, r = 3, 8, 12, 4
    area = rng.uniform(1, 2, (ny, nx))
    c = 7.25
    m, W = C.coarse_grain_mean(np.full((nz, ny, nx), c), np.broadcast_to(area, (nz, ny, nx)), r)
    assert np.allclose(m, c, rtol=1e-15)
    assert np.allclose(W[0], area.reshape(2, 4, 3, 4).sum(axis=(1, 3)))
    # a tracer constant within each block carries no subgrid flux, whatever w does
    Tb = rng.normal(size=(nz, ny // r, nx // r))
    T = np.repeat(np.repeat(Tb, r, axis=1), r, axis=2)
    T[1:] = T[1:] * 0 + T[:1]                     # and uniform in depth, so T_f is exact
    w = rng.normal(size=(nz, ny, nx))
    kb = np.zeros((ny, nx), dtype=int)
    F = C.subgrid_vertical_flux(w, T, kb, area, r)
    assert np.max(np.abs(F)) < 1e-13
    # w = a + b T' inside a block gives <wT> - <w><T> = b var(T) exactly
    T = rng.normal(size=(nz, ny, nx))
    T[:] = T[:1]
    w = 0.3 + 2.0 * T
    F = C.subgrid_vertical_flux(w, T, kb, np.ones((ny, nx)), r)
    var = T[0].reshape(2, 4, 3, 4).var(axis=(1, 3))
    np.testing.assert_allclose(F[1], 2.0 * var, rtol=1e-12)
    assert np.all(F[0] == 0.0)
