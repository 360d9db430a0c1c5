"""The closure network's tensor-core kernels against the FP64 oracle (needs a GPU):
forward outputs and loss gradients on bfloat16-exact weights and inputs, and training
that lowers the loss."""
import numpy as np
import pytest

from oracle import closure as C
from paper_2309_06662_gb300 import inputs, ocean

pytestmark = pytest.mark.gpu

SCALES = dict(kappa=1e-2, gT=1e-6, gS=1e-7, sFT=1e-5, sFS=1e-6, sGT=1e-6, sGS=1e-7)


def _cos(a, b):
    a, b = a.ravel(), b.ravel()
    return float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-300))


def _data(nz, M, seed):
    rng = np.random.default_rng(seed)
    X = C.bf16_round(rng.normal(size=(M, 6 * nz)))
    d = dict(dzT=rng.normal(0, 1e-3, (M, nz)), dzS=rng.normal(0, 1e-4, (M, nz)),
             FT=rng.normal(0, 1e-5, (M, nz)), FS=rng.normal(0, 1e-6, (M, nz)),
             GT=rng.normal(0, 1e-6, (M, nz)), GS=rng.normal(0, 1e-7, (M, nz)))
    face = rng.random((M, nz)) > 0.2
    wet = rng.random((M, nz)) > 0.1
    return X, d, face, wet


def _torch_batch(X, d, face, wet):
    import torch
    t = {k: torch.tensor(v, dtype=torch.float32, device="cuda") for k, v in d.items()}
    t["X"] = torch.tensor(X, dtype=torch.float32, device="cuda")
    t["face"] = torch.tensor(face.astype(np.uint8), device="cuda")
    t["wet"] = torch.tensor(wet.astype(np.uint8), device="cuda")
    return t


@pytest.mark.parametrize("nz,hidden,M", [(48, 256, 512), (8, 32, 136)])
def test_forward_matches_oracle(nz, hidden, M):
    import torch
    params = inputs.mlp_seeded_params(7, [6 * nz, hidden, hidden, hidden, 3 * nz])
    X, _, _, _ = _data(nz, M, 1)
    net = ocean.MLP(nz, hidden, M, params)
    Y = net.forward(torch.tensor(X, dtype=torch.float32)).cpu().double().numpy()
    ref, _ = C.mlp_forward(params, X, bf16=True)
    err = np.linalg.norm(Y - ref) / np.linalg.norm(ref)
    assert err < 1e-2 and _cos(Y, ref) > 0.9999, err
    # parameters round-trip through the handle unchanged
    for (W, b), (W2, b2) in zip(params, net.get_params()):
        assert np.array_equal(W, W2) and np.array_equal(b, b2)


def test_loss_and_gradients_match_oracle():
    nz, hidden, M = 48, 256, 1024
    params = inputs.mlp_seeded_params(11, [6 * nz, hidden, hidden, hidden, 3 * nz])
    X, d, face, wet = _data(nz, M, 2)
    net = ocean.MLP(nz, hidden, M, params)
    loss, grads = net.loss_grad(_torch_batch(X, d, face, wet), SCALES)
    Y, cache = C.mlp_forward(params, X, bf16=True)
    L, dY = C.closure_loss(Y, nz, SCALES, d["dzT"], d["dzS"], d["FT"], d["FS"], d["GT"], d["GS"],
                           face, wet)
    ref = C.mlp_backward(params, cache, dY, bf16=True)
    assert abs(loss - L) <= 1e-2 * abs(L)
    for li, ((gW, gb), (rW, rb)) in enumerate(zip(grads, ref)):
        for g, r in ((gW, rW), (gb, rb)):
            rel = np.linalg.norm(g - r) / np.linalg.norm(r)
            assert rel < 1e-2 and _cos(g, r) > 0.9999, (li, rel, _cos(g, r))


def test_training_lowers_the_loss():
    nz, hidden, M = 16, 64, 2048
    params = inputs.mlp_seeded_params(3, [6 * nz, hidden, hidden, hidden, 3 * nz])
    X, d, face, wet = _data(nz, M, 5)
    # every target a fixed function of the inputs (a constant diffusivity of half the
    # scale for both fluxes, bounded functions of T and S for the tendencies)
    d["FT"] = -1e-2 * 0.5 * d["dzT"]
    d["FS"] = -1e-2 * 0.5 * d["dzS"]
    d["GT"] = 1e-6 * np.tanh(X[:, :nz])
    d["GS"] = 1e-7 * np.tanh(X[:, nz:2 * nz])
    t = _torch_batch(X, d, face, wet)
    net = ocean.MLP(nz, hidden, M, params)
    l0 = net.train_step(t, SCALES, 1e-3)
    for _ in range(300):
        l1 = net.train_step(t, SCALES, 1e-3)
    assert l1 < 0.1 * l0, (l0, l1)
