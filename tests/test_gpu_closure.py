"""The closure network's tensor-core kernels against the FP64 oracle (needs a GPU):
forward outputs and loss gradients on bfloat16-exact weights and inputs, and training
that lowers the loss."""
import ctypes

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


def test_adam_steps_match_oracle_elementwise():
    # three Adam steps of the trainer handle against oracle adam_step applied to the GPU's
    # own gradients (taken at the GPU's current weights before each step): the FP32
    # master weights agree to FP32 rounding (the update is lr times a ratio of moments,
    # so a wrong bias correction, beta or epsilon shows at the lr scale), and the BF16
    # copies the GEMMs read are the rounding of those weights (the forward pass of the
    # handle equals the oracle forward of its own weights)
    import torch
    nz, hidden, M = 8, 32, 256
    dims = [6 * nz, hidden, hidden, hidden, 3 * nz]
    params = inputs.mlp_seeded_params(13, dims)
    X, d, face, wet = _data(nz, M, 9)
    t = _torch_batch(X, d, face, wet)
    net = ocean.MLP(nz, hidden, M, params)
    w = [[W.astype(np.float64).copy(), b.astype(np.float64).copy()] for W, b in params]
    mom = [[np.zeros_like(W), np.zeros_like(b)] for W, b in w]
    vel = [[np.zeros_like(W), np.zeros_like(b)] for W, b in w]
    lr = 1e-3
    for step in (1, 2, 3):
        _, grads = net.loss_grad(t, SCALES)
        net.train_step(t, SCALES, lr)
        for li in range(4):
            for q in range(2):
                C.adam_step(w[li][q], grads[li][q], mom[li][q], vel[li][q], step, lr=lr)
        got = net.get_params()
        for li in range(4):
            for q in range(2):
                diff = np.abs(got[li][q] - w[li][q])
                bound = 4e-7 * np.abs(w[li][q]) + 1e-5 * lr
                assert np.all(diff <= bound), (step, li, q, float(np.max(diff / bound)))
    Y = net.forward(torch.tensor(X, dtype=torch.float32)).cpu().double().numpy()
    ref, _ = C.mlp_forward(net.get_params(), X, bf16=True)
    err = np.linalg.norm(Y - ref) / np.linalg.norm(ref)
    assert err < 1e-2 and _cos(Y, ref) > 0.9999, err


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


# ----------------------------------------------------------------------------- in the model

import oracle  # noqa: E402
from tests.oracle_cases import seeded_velocity  # noqa: E402


def _stats(raw, msk):
    mu = np.array([raw[msk[:, f], f].mean() if msk[:, f].any() else 0.0 for f in range(raw.shape[1])])
    sd = np.array([raw[msk[:, f], f].std() if msk[:, f].any() else 1.0 for f in range(raw.shape[1])])
    return mu, np.where(sd > 0, sd, 1.0)


def _oracle_features(o, c):
    p = c.params
    return C.column_features(o.get("T"), o.get("S"), o.get("u"), o.get("v"), o.kb_array(),
                             np.asarray(c.z_faces), p["g"], p["alpha"], p["beta_s"],
                             bool(c.periodic_x), bool(c.periodic_y))


def test_features_match_oracle():
    c = inputs.latlon_small_case(seed=21)
    c.u, c.v = seeded_velocity(c, 6, 0.05)
    o = oracle.OracleModel(c)
    raw, msk = _oracle_features(o, c)
    mu, sd = _stats(raw, msk)
    g = ocean.Ocean(c, precision=ocean.OCEAN_FP64)
    f = g.closure_features(mu, sd)
    X = f["X"].cpu().double().numpy()
    ref = C.normalise(raw, msk, mu, sd)
    assert np.max(np.abs(X - ref)) <= 1e-5 * np.max(np.abs(ref))
    nz = c.nz
    assert np.array_equal(f["wet"].cpu().numpy().astype(bool), msk[:, :nz])
    assert np.array_equal(f["face"].cpu().numpy().astype(bool), msk[:, 4 * nz:5 * nz])


def _pair():
    fine, coarse = inputs.latlon_pair(18, 10, 8, 70.0, 4, seed=8, dt_coarse=1800.0, ns_coarse=20,
                                      ns_fine=20, corr_deg=20.0)
    fine.u, fine.v = seeded_velocity(fine, 9, 0.05)
    fine.eta = 0.1 * inputs.random_normal(8, 30, fine.nx * fine.ny).reshape(fine.ny, fine.nx)
    return fine, coarse


def test_coarse_grain_and_targets_match_oracle():
    fine, coarse = _pair()
    r = 4
    # GPU
    gf = ocean.Ocean(fine, precision=ocean.OCEAN_FP64)
    gc = ocean.Ocean(coarse, precision=ocean.OCEAN_FP64)
    gc.set_reference(*gf.get_reference())
    gf.tendencies()
    t = gf.coarse_grain_to(gc, r)
    gc.tendencies()
    gc.closure_targets(t)
    # oracle, from the same seeded fine state
    of = oracle.OracleModel(fine)
    of.tendencies()
    oc = oracle.OracleModel(coarse)
    st = {k: of.get(k) for k in ("u", "v", "T", "S", "w", "eta")}
    st["GT"], st["GS"] = of.get("GT"), of.get("GS")
    area = inputs.latlon_row_area(fine.ny, 70.0, fine.nx)
    out, FT, FS, GTm, GSm = C.coarse_grain_state(st, of.kb_array(), oc.kb_array(), area, r)
    for f in ("u", "v", "T", "S", "eta"):
        a, b = gc.get(f), out[f]
        assert np.max(np.abs(a - b)) <= 1e-10 * max(1e-30, np.max(np.abs(b))), f
    flat = lambda A: A.reshape(A.shape[0], -1).T
    for name, ref in (("FT", FT), ("FS", FS), ("GTm", GTm), ("GSm", GSm)):
        got = t[name].cpu().double().numpy()
        assert np.max(np.abs(got - flat(ref))) <= 1e-5 * max(1e-30, np.max(np.abs(ref))), name
    # lateral residual targets from the oracle's own coarse model on its coarse state
    for f in ("u", "v", "T", "S", "eta"):
        oc.set(f, out[f])
    oc.tendencies()
    dz = np.diff(np.asarray(coarse.z_faces))
    FTu = np.concatenate([FT[1:], np.zeros((1,) + FT.shape[1:])])
    ref = np.where(flat(GTm) != 0, flat(GTm - oc.get("GT") + (FTu - FT) / dz[:, None, None]), 0.0)
    got = t["GT"].cpu().double().numpy()
    wet = flat(np.arange(coarse.nz)[:, None, None] >= oc.kb_array()[None])
    assert np.max(np.abs((got - ref)[wet])) <= 1e-4 * np.max(np.abs(ref[wet]))


@pytest.mark.parametrize("precision,tol", [(ocean.OCEAN_FP64, 1e-6), (ocean.OCEAN_MIXED, 2e-4)])
def test_learned_step_matches_oracle(precision, tol):
    c = inputs.latlon_small_case(seed=23)
    c.u, c.v = seeded_velocity(c, 7, 0.05)
    nz, hidden = c.nz, 32
    o = oracle.OracleModel(c)
    mu, sd = _stats(*_oracle_features(o, c))
    params = inputs.mlp_seeded_params(19, [6 * nz, hidden, hidden, hidden, 3 * nz])
    sc = dict(kappa=2e-3, gT=2e-8, gS=2e-9, sFT=1, sFS=1, sGT=1, sGS=1)
    g = ocean.Ocean(c, precision=precision, closure=ocean.OCEAN_CLOSURE_LEARNED,
                    closure_hidden=hidden)
    g.set_closure(params, mu, sd, sc)
    g.step(5)
    C.step_learned(o, 5, params, mu, sd, sc, bf16=True)
    for f in ("u", "v", "T", "S", "eta"):
        a, b = g.get(f), o.get(f)
        err = np.linalg.norm(a - b) / np.linalg.norm(b)
        assert err <= tol, (f, err)
    # and the closure changed the answer: on the temperature anomaly T - T(0), where the
    # closure acts, the plain step is far further from the learned oracle than the GPU is
    p = oracle.OracleModel(c)
    p.step(5)
    wet = o.get("T") != 0
    anom = lambda m: (m.get("T") - np.asarray(c.T))[wet]
    ref = np.linalg.norm(anom(o))
    effect = np.linalg.norm(anom(p) - anom(o)) / ref
    err = np.linalg.norm(anom(g) - anom(o)) / ref
    assert effect > 1e-3, effect
    assert err < 0.05 * effect, (err, effect)


@pytest.mark.gpu
def test_bounded_wait_gives_up_and_the_context_survives():
    # a device wait on a barrier that nothing completes returns OCEAN_ERR_TIMEOUT (no
    # hang, no trap); the GEMM kernels use the same wait, and still run afterwards
    import torch
    L = ocean.load()
    s = torch.cuda.current_stream().cuda_stream
    rc = L.ocean_selftest_bounded_wait(2_000_000, ctypes.c_void_p(s))
    assert rc == -4, rc
    assert b"gave up" in L.ocean_last_error(None)
    nz, H, M = 4, 32, 64
    dims = [6 * nz, H, H, H, 3 * nz]
    params = inputs.mlp_seeded_params(3, dims)
    net = ocean.MLP(nz, H, M, params)
    X = torch.tensor(np.random.default_rng(1).normal(size=(M, 6 * nz)), dtype=torch.float32,
                     device="cuda")
    Y = net.forward(X).cpu().numpy()
    ref, _ = C.mlp_forward(params, X.cpu().numpy().astype(np.float64), bf16=True)
    assert np.max(np.abs(Y - ref)) <= 1e-2 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.gpu
@pytest.mark.parametrize("bad_output", [0, 5, 7, 100])
def test_columns_with_a_non_finite_output_keep_the_richardson_closure(bad_output):
    # one output of the network made NaN for every column (through the last layer's
    # bias): no column's outputs are applied, so the learned step is bitwise the
    # Richardson-number step.  The output's index decides which of the threads that
    # test a column's outputs sees it.
    c = inputs.latlon_small_case(seed=23)
    c.u, c.v = seeded_velocity(c, 7, 0.05)
    nz, hidden = c.nz, 32
    o = oracle.OracleModel(c)
    mu, sd = _stats(*_oracle_features(o, c))
    params = inputs.mlp_seeded_params(19, [6 * nz, hidden, hidden, hidden, 3 * nz])
    W, b = params[-1]
    b = np.array(b, dtype=np.float64, copy=True)
    b[bad_output % (3 * nz)] = np.nan
    params = params[:-1] + [(W, b)]
    sc = dict(kappa=2e-3, gT=2e-8, gS=2e-9, sFT=1, sFS=1, sGT=1, sGS=1)
    g = ocean.Ocean(c, precision=ocean.OCEAN_MIXED, closure=ocean.OCEAN_CLOSURE_LEARNED,
                    closure_hidden=hidden)
    g.set_closure(params, mu, sd, sc)
    r = ocean.Ocean(c, precision=ocean.OCEAN_MIXED)
    g.step(3)
    r.step(3)
    for f in ("u", "v", "T", "S", "eta"):
        assert np.array_equal(g.get(f), r.get(f)), f
