"""Train and evaluate the learned column closure against coarse-grained fine runs.

    python -m paper_2309_06662_gb300.closure_train --config half --out closure.json

1. Training data: fine runs (r times finer in x and y, time step dt/r, the same seeded
   recipe; one per training seed) are advanced over the same span of time as the
   evaluation below and, every `snap_every` fine steps, coarse-grained onto the coarse
   grid (ocean_coarse_grain).
   The coarse state gives the network inputs (ocean_closure_features); the fine fields
   give the subgrid vertical fluxes <w T> - <w><T> and, with the coarse model's own
   tendencies, the lateral residual targets (ocean_closure_targets).
2. Training: z-scored inputs, Adam on the normalised closure loss with this library's
   BF16 tensor-core forward and backward kernels (ocean_mlp_train_step).  The columns
   of the easternmost `val_frac` of the domain are held back for validation (other
   bathymetry than the training columns); the weights of the epoch with the lowest
   validation loss are kept, and an output head (the diffusivity, or the two tendency
   corrections) that does not beat "no network" on the validation columns is switched
   off (diffusivity head: softplus(-30), i.e. no extra diffusivity; correction head: 0).
3. A priori: on coarse-grained snapshots of a second fine run (another seed), the loss
   of the trained network against that of the Richardson-number closure alone.  The
   network's diffusivity is added to the Richardson-number one, so "alone" means zero
   extra diffusivity and no tendency correction.
4. Online: coarse runs with each closure from the coarse-grained state of that second
   run, compared with its later coarse-grained states (T, S root-mean-square over wet
   cells) at matched times, and the cost of a step with each.

Everything runs on the GPU through the C ABI; torch only holds device arrays, shuffles
the training set and reduces statistics.
"""
from __future__ import annotations

import argparse
import json
import math
import time
from typing import Dict

import numpy as np

from . import inputs, ocean

CONFIGS = {
    # the 1/2-degree coarse grid (720 x 320 x 48, 80S-80N) and its 1/8-degree fine run
    # (2880 x 1280 x 48); 480 s and 120 s keep the explicit internal-wave step stable at
    # the 2.4 km zonal spacing next to 80 degrees (at 150 s the fine run diverges); 16
    # snapshots over the 8800 fine steps the evaluation spans, ~2.6M columns
    "half": dict(nxc=720, nyc=320, nz=48, lat=80.0, r=4, dt=480.0, ns_coarse=60, ns_fine=60,
                 train_seeds=(5,), eval_seed=4, snaps=16, snap_every=550, val_frac=0.125,
                 spinup=800, eval_steps=2000, check_every=250, epochs=20, batch=4096,
                 hidden=256, lr=1e-3, kappa=1e-3),
    # a seconds-long version of the same pipeline (tests): 176 fine steps evaluated, four
    # training runs
    "small": dict(nxc=36, nyc=16, nz=8, lat=70.0, r=4, dt=1800.0, ns_coarse=20, ns_fine=20,
                  train_seeds=(5, 6, 7, 8), eval_seed=4, snaps=22, snap_every=8,
                  val_frac=0.25, spinup=16, eval_steps=40, check_every=20, epochs=60,
                  batch=128, hidden=32, lr=2e-3, kappa=1e-3),
}


def fine_model(cfg: Dict, seed: int):
    """The fine model of the pair (and the matching coarse case) for one seed."""
    fine_c, coarse_c = inputs.latlon_pair(cfg["nxc"], cfg["nyc"], cfg["nz"], cfg["lat"],
                                          cfg["r"], seed, cfg["dt"], cfg["ns_coarse"],
                                          cfg["ns_fine"])
    return ocean.Ocean(fine_c, precision=ocean.OCEAN_MIXED), coarse_c


def coarse_model(coarse_c, fine, hidden: int = 0):
    """A mixed-precision coarse model sharing the fine model's reference profiles, so
    that coarse-grained anomalies are anomalies of the coarse model too."""
    closure = ocean.OCEAN_CLOSURE_LEARNED if hidden else ocean.OCEAN_CLOSURE_RI
    m = ocean.Ocean(coarse_c, precision=ocean.OCEAN_MIXED, closure=closure,
                    closure_hidden=hidden)
    m.set_reference(*fine.get_reference())
    return m


def check_finite(model, what: str) -> None:
    """Raise if the model's state is no longer finite."""
    d = model.diagnostics()
    if d["nonfinite"]:
        raise RuntimeError(f"{what}: the state is not finite at step {d['step']} "
                           f"(max CFL {d['max_cfl']:.3g})")


def snapshot(fine, coarse, r: int):
    """Coarse-grain the fine state onto `coarse` (replacing its state) and return the raw
    network inputs, masks and targets of its wet columns (torch CUDA tensors) and their
    column indices."""
    import torch
    check_finite(fine, "fine run")
    fine.tendencies()
    t = fine.coarse_grain_to(coarse, r)
    coarse.tendencies()
    coarse.closure_targets(t)
    nz = coarse.nz
    f = coarse.closure_features(np.zeros(6 * nz), np.ones(6 * nz))
    keep = f["wet"].bool().any(dim=1)
    out = dict(X=f["X"], face=f["face"], wet=f["wet"], dzT=f["dzT"], dzS=f["dzS"],
               FT=t["FT"], FS=t["FS"], GT=t["GT"], GS=t["GS"])
    out = {k: v[keep].contiguous() for k, v in out.items()}
    cols = torch.arange(keep.numel(), device="cuda")[keep]
    return out, cols


def split_east(d, cols, nx: int, frac: float):
    """(rest, east): the columns of the easternmost `frac` of the domain apart."""
    east = (cols % nx) >= int(round(nx * (1.0 - frac)))
    return ({k: v[~east].contiguous() for k, v in d.items()},
            {k: v[east].contiguous() for k, v in d.items()})


def concat(parts):
    """Concatenate per-snapshot training tensors along the column axis."""
    import torch
    return {k: torch.cat([p[k] for p in parts]).contiguous() for k in parts[0]}


def pad8(d):
    """Pad a set to a multiple of 8 columns with columns that count nowhere."""
    import torch
    n = d["X"].shape[0]
    extra = (-n) % 8
    if not extra:
        return d
    return {k: torch.cat([v, torch.zeros((extra,) + tuple(v.shape[1:]), dtype=v.dtype,
                                         device=v.device)]).contiguous() for k, v in d.items()}


def _feature_mask(d):
    import torch
    return torch.cat([d["wet"]] * 4 + [d["face"]] * 2, dim=1).bool()


def feature_stats(d):
    """Per-feature mean and standard deviation over the entries that count (wet levels
    for T, S, u, v; interior faces for N^2, shear^2); sigma 1 where a feature is flat."""
    import torch
    X, mask = d["X"].double(), _feature_mask(d)
    cnt = mask.sum(0).clamp(min=1).double()
    mu = (X * mask).sum(0) / cnt
    sd = ((((X - mu) * mask) ** 2).sum(0) / cnt).sqrt()
    sd = torch.where(sd > 0, sd, torch.ones_like(sd))
    return mu.cpu().numpy(), sd.cpu().numpy()


def normalise(d, mu, sd):
    """z-score the features of a training set with the given statistics."""
    import torch
    m = torch.tensor(mu, dtype=torch.float32, device="cuda")
    s = torch.tensor(sd, dtype=torch.float32, device="cuda")
    d["X"] = torch.where(_feature_mask(d), (d["X"] - m) / s,
                         torch.zeros((), device="cuda")).contiguous()
    return d


def target_scales(d, kappa: float) -> Dict[str, float]:
    """Output scales (kappa, dG_T, dG_S) and loss normalisations from the training set:
    each target's standard deviation over its entries."""
    def sd(x, m):
        v = x[m.bool()].double()
        s = float(v.std().item()) if v.numel() > 1 else 0.0
        return s if s > 0 else 1.0
    sGT, sGS = sd(d["GT"], d["wet"]), sd(d["GS"], d["wet"])
    return dict(kappa=kappa, gT=sGT, gS=sGS, sFT=sd(d["FT"], d["face"]),
                sFS=sd(d["FS"], d["face"]), sGT=sGT, sGS=sGS)


def baseline_loss(d, sc) -> float:
    """The closure loss with no network: zero extra diffusivity, no correction."""
    face, wet = d["face"].bool(), d["wet"].bool()
    nf, nw = max(1, int(face.sum())), max(1, int(wet.sum()))
    q = lambda x, m, s: float(((x[m].double() / s) ** 2).sum())
    return ((q(d["FT"], face, sc["sFT"]) + q(d["FS"], face, sc["sFS"])) / nf
            + (q(d["GT"], wet, sc["sGT"]) + q(d["GS"], wet, sc["sGS"])) / nw)


def loss_terms(Y, d, sc) -> Dict[str, float]:
    """The four normalised terms of the closure loss (vertical T and S fluxes on faces,
    T and S corrections on wet levels) for network outputs Y; Y = None: no network."""
    import torch
    face, wet = d["face"].bool(), d["wet"].bool()
    nz = face.shape[1]
    nf, nw = max(1, int(face.sum())), max(1, int(wet.sum()))
    if Y is None:
        kap = torch.zeros_like(d["FT"], dtype=torch.float64)
        gT = gS = kap
    else:
        Y = Y.double()
        kap = sc["kappa"] * torch.nn.functional.softplus(Y[:, :nz])
        gT, gS = sc["gT"] * Y[:, nz:2 * nz], sc["gS"] * Y[:, 2 * nz:]
    q = lambda r, m, n: float((r[m] ** 2).sum()) / n
    return dict(fT=q((-kap * d["dzT"].double() - d["FT"].double()) / sc["sFT"], face, nf),
                fS=q((-kap * d["dzS"].double() - d["FS"].double()) / sc["sFS"], face, nf),
                gT=q((gT - d["GT"].double()) / sc["sGT"], wet, nw),
                gS=q((gS - d["GS"].double()) / sc["sGS"], wet, nw))


def train(net, d, sc, epochs: int, batch: int, lr: float, val=None, ev=None, seed: int = 0):
    """Adam over shuffled batches.  Returns the mean batch loss of each epoch, the
    validation loss after each epoch (with `val` and an evaluation handle `ev` that
    holds the whole validation set), the parameters of the best epoch and its validation
    loss terms."""
    import torch
    n = d["X"].shape[0]
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    hist, vhist, best, best_v, best_terms = [], [], None, math.inf, None
    for _ in range(epochs):
        perm = torch.randperm(n, device="cuda", generator=g)
        tot, cnt = 0.0, 0
        for a in range(0, n - batch + 1, batch):
            idx = perm[a:a + batch]
            part = {k: v.index_select(0, idx).contiguous() for k, v in d.items()}
            tot += net.train_step(part, sc, lr)
            cnt += 1
        hist.append(tot / max(1, cnt))
        if val is not None:
            params = net.get_params()
            ev.set_params(params)
            vl = ev.loss_grad(val, sc, grads=False)[0]
            vhist.append(vl)
            if vl < best_v:
                best, best_v = params, vl
                best_terms = loss_terms(ev.forward(val["X"]), val, sc)
    if best is None:
        best = net.get_params()
    return hist, vhist, best, best_terms


def gate_heads(params, nz: int, terms, base, corrections: bool = True):
    """Switch off the output heads that do not beat "no network" on validation columns
    (and the correction head when it was not fitted): returns the gated parameters and
    which heads stay on."""
    W, b = (x.copy() for x in params[-1])
    # the correction head must beat zero by 2%: kept on a hair's margin at 1/2 degree it
    # forced the coarse run to non-finite values within 750 steps
    keep = dict(diffusivity=terms["fT"] + terms["fS"] < base["fT"] + base["fS"],
                corrections=corrections
                and terms["gT"] + terms["gS"] < 0.98 * (base["gT"] + base["gS"]))
    if not keep["diffusivity"]:
        W[:, :nz] = 0.0
        b[:nz] = -30.0
    if not keep["corrections"]:
        W[:, nz:] = 0.0
        b[nz:] = 0.0
    return params[:-1] + [(W, b)], keep


def fmt_terms(t) -> str:
    """The four loss terms (fT, fS, gT, gS) as one short string."""
    return "/".join(f"{t[k]:.3g}" for k in ("fT", "fS", "gT", "gS"))


def wet_rms(a: np.ndarray, b: np.ndarray, wet: np.ndarray) -> float:
    """Root-mean-square difference of two fields over the wet cells."""
    return float(np.sqrt(np.mean((a - b)[wet] ** 2)))


def run(cfg: Dict, log=print) -> Dict:
    """The whole pipeline for one configuration: fine runs, coarse-grained targets,
    training with a held-out longitude band, a priori evaluation on another seed and
    online runs of the coarse model with and without the network; returns the results."""
    import torch
    r, nz, H = cfg["r"], cfg["nz"], cfg["hidden"]
    t0 = time.time()
    # ------------------------------------------------------------------ training data
    parts, vparts = [], []
    for seed in cfg["train_seeds"]:
        fine, coarse_c = fine_model(cfg, seed)
        coarse = coarse_model(coarse_c, fine)
        for _ in range(cfg["snaps"]):
            fine.step(cfg["snap_every"])
            tr, va = split_east(*snapshot(fine, coarse, r), cfg["nxc"], cfg["val_frac"])
            parts.append(tr)
            vparts.append(va)
        fine.close()
        coarse.close()
    data, val = concat(parts), concat(vparts)
    del parts, vparts
    mu, sd = feature_stats(data)
    normalise(data, mu, sd)
    val = pad8(normalise(val, mu, sd))
    sc = target_scales(data, cfg["kappa"])
    ncols = int(data["X"].shape[0])
    log(f"training set: {ncols} columns, validation {int(val['X'].shape[0])} "
        f"({time.time() - t0:.1f} s)")
    # ------------------------------------------------------------------ training
    dims = [6 * nz, H, H, H, 3 * nz]
    net = ocean.MLP(nz, H, cfg["batch"], inputs.mlp_seeded_params(cfg["train_seeds"][0], dims))
    vev = ocean.MLP(nz, H, val["X"].shape[0])
    # fit_corrections = False: the tendency-correction terms leave the training loss (their
    # normalisation made huge), so the shared layers serve the diffusivity alone and the
    # correction head stays off; the training and validation losses are those of tsc
    fit_corr = cfg.get("fit_corrections", True)
    tsc = dict(sc) if fit_corr else dict(sc, sGT=1e30, sGS=1e30)
    train_base = baseline_loss(data, tsc)
    val_base = baseline_loss(val, tsc)
    torch.cuda.synchronize()
    t1 = time.time()
    hist, vhist, trained, _ = train(net, data, tsc, cfg["epochs"], cfg["batch"], cfg["lr"],
                                    val, vev, seed=cfg.get("train_seed", 0))
    torch.cuda.synchronize()
    train_s = time.time() - t1
    vev.set_params(trained)
    vterms = loss_terms(vev.forward(val["X"]), val, sc)
    vbase_terms = loss_terms(None, val, sc)
    trained, heads = gate_heads(trained, nz, vterms, vbase_terms, corrections=fit_corr)
    steps = cfg["epochs"] * (ncols // cfg["batch"])
    log(f"training: {steps} Adam steps in {train_s:.1f} s, loss {hist[0]:.4g} -> {hist[-1]:.4g}"
        f" (no network: {train_base:.4g}); validation best {min(vhist):.4g} at epoch "
        f"{vhist.index(min(vhist)) + 1} (no network: {val_base:.4g}); validation terms "
        f"{fmt_terms(vterms)} vs {fmt_terms(vbase_terms)}; heads kept: {heads}")
    del data, val
    net.close()
    vev.close()
    # ------------------------------------------------------------------ held-out run
    fine, coarse_c = fine_model(cfg, cfg["eval_seed"])
    ref = coarse_model(coarse_c, fine)
    fine.step(cfg["spinup"])
    held = pad8(normalise(snapshot(fine, ref, r)[0], mu, sd))
    # one evaluation handle holding a whole snapshot: the loss of one call is exact
    ev = ocean.MLP(nz, H, held["X"].shape[0], trained)

    def assess(step, d):
        return dict(step=step, learned=ev.loss_grad(d, sc, grads=False)[0],
                    richardson=baseline_loss(d, sc), terms_learned=loss_terms(ev.forward(d["X"]), d, sc),
                    terms_richardson=loss_terms(None, d, sc))

    apriori = [assess(0, held)]
    ri = coarse_model(coarse_c, fine)
    ml = coarse_model(coarse_c, fine, hidden=H)
    ml.set_closure(trained, mu, sd, sc)
    for m in (ri, ml):      # the same coarse-grained start
        fine.coarse_grain_to(m, r)
    wet = ref.closure_features()["wet"].bool().T.reshape(nz, cfg["nyc"], cfg["nxc"]).cpu().numpy()
    online, cost, done = [], {"richardson": 0.0, "learned": 0.0}, 0
    while done < cfg["eval_steps"]:
        n = min(cfg["check_every"], cfg["eval_steps"] - done)
        for name, m in (("richardson", ri), ("learned", ml)):
            torch.cuda.synchronize()
            a = time.perf_counter()
            m.step(n)
            torch.cuda.synchronize()
            cost[name] += time.perf_counter() - a
        done += n
        fine.step(r * n)
        held = pad8(normalise(snapshot(fine, ref, r)[0], mu, sd))
        apriori.append(assess(done, held))
        Tr, Sr = ref.get("T"), ref.get("S")
        row = dict(step=done)
        for name, m in (("richardson", ri), ("learned", ml)):
            row["rms_T_" + name] = wet_rms(m.get("T"), Tr, wet)
            row["rms_S_" + name] = wet_rms(m.get("S"), Sr, wet)
            row["finite_" + name] = not m.diagnostics()["nonfinite"]
        online.append(row)
        a = apriori[-1]
        log(f"step {done}: a priori loss learned {a['learned']:.4g} vs {a['richardson']:.4g} "
            f"(terms {fmt_terms(a['terms_learned'])} vs {fmt_terms(a['terms_richardson'])}); "
            f"RMS T Ri {row['rms_T_richardson']:.4g} "
            f"learned {row['rms_T_learned']:.4g}; RMS S Ri {row['rms_S_richardson']:.4g} "
            f"learned {row['rms_S_learned']:.4g}")
    for m in (fine, ref, ri, ml, ev):
        m.close()
    return dict(config=cfg, training_columns=ncols, scales=sc, loss_history=hist,
                validation_history=vhist, validation_baseline=val_base,
                validation_terms=vterms, validation_terms_baseline=vbase_terms, heads=heads,
                training_baseline=train_base, train_seconds=train_s, adam_steps=steps,
                apriori=apriori, online=online,
                ms_per_step={k: 1e3 * v / max(1, done) for k, v in cost.items()})


def main():
    """Command line: run one configuration and print (or write) its results."""
    ap = argparse.ArgumentParser(description="Train and evaluate the learned closure.")
    ap.add_argument("--config", choices=sorted(CONFIGS), default="half")
    ap.add_argument("--out", default=None, help="write the results as JSON")
    ap.add_argument("--epochs", type=int, default=None)
    ap.add_argument("--eval-steps", type=int, default=None)
    ap.add_argument("--lr", type=float, default=None)
    args = ap.parse_args()
    cfg = dict(CONFIGS[args.config])
    if args.epochs is not None:
        cfg["epochs"] = args.epochs
    if args.eval_steps is not None:
        cfg["eval_steps"] = args.eval_steps
    if args.lr is not None:
        cfg["lr"] = args.lr
    res = run(cfg)
    if args.out:
        with open(args.out, "w") as f:
            json.dump(res, f, indent=1)
    print(json.dumps({k: res[k] for k in ("training_columns", "train_seconds", "ms_per_step")}))


if __name__ == "__main__":
    main()
