"""Learned repair-strategy selector: label collection, training and use.

The selector has no counterpart in the paper.  It learns the repair/rebuild
crossover whose shape Prop. 1 describes and whose location Sec. 4 measures.
It never changes a certificate, only which exact strategy runs.

* Features: eight per scene and step, computed on the device by the step
  itself (``Context.features``; definitions in include/cert.h).
* Labels: ln of the measured step time of incremental repair and of rebuild,
  both timed with CUDA events from identical state (``cert_snapshot`` /
  ``cert_restore``).  In training rows, feature 8 is replaced by the measured
  previous ln(t_inc / t_reb).
* Network: MLP 8-64-64-2, ReLU, MSE on the log times, Adam.  Forward, backward
  and Adam all run in the library's kernels (``cert_mlp_*``); this module only
  slices minibatches and moves arrays.
* Decision: incremental when ln t_inc - ln t_reb <= delta, the margin with the
  least regret on the training rows (``decision_margin``), folded into the
  rebuild head's bias so the in-loop argmin applies it.

CLI (on a GPU):
    python -m paper_2606_18314_b300.selector collect --out labels.npz [--seeds 16]
    python -m paper_2606_18314_b300.selector train --data labels.npz --out selector_weights.npz
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

from . import scenes

HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(HERE, "selector_weights.npz")
N_FEAT = 8
FEATURES = ["frontier_frac", "H_cand", "ln_N", "dim", "ln1p_eps_over_med_c", "touched_cell_frac",
            "prev_fail_ratio", "prev_ln_time_ratio"]
LAYOUT = [("W1", (64, 8)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)), ("W3", (2, 64)), ("b3", (2,))]


def he_init(seed: int) -> np.ndarray:
    """He-normal weights, zero biases, flat in the library's layout."""
    r = np.random.Generator(np.random.Philox(np.random.SeedSequence([7, seed])))
    parts = []
    for name, shp in LAYOUT:
        if name.startswith("W"):
            parts.append(r.standard_normal(shp) * math.sqrt(2.0 / shp[1]))
        else:
            parts.append(np.zeros(shp))
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32)


def normalisation(X: np.ndarray) -> np.ndarray:
    """mean[8] then 1/std[8] of the training features (std floored at 1e-6)."""
    mu = X.mean(axis=0)
    sd = np.maximum(X.std(axis=0), 1e-6)
    return np.concatenate([mu, 1.0 / sd]).astype(np.float32)


# ----------------------------------------------------------------------------- labels

def time_step(ctx, pos, eps, strategy, torch):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    ctx.step(pos, eps, strategy)
    e1.record()
    e1.synchronize()
    return e0.elapsed_time(e1)


def collect_trajectory(frames, eps, offsets=None, torch=None):
    """Both strategies timed from identical state at every step of a
    trajectory.  Returns (X [steps][scenes*8], T [steps][2] ln ms).  With
    several scenes the features of scene 0 are kept (single-scene use)."""
    from . import cert
    dev = torch.from_numpy(frames).cuda()
    ctx = cert.Context(dev[0], offsets=offsets)
    X, T = [], []
    prev_ratio = 0.0
    # one untimed warm step so that kernels and the grid are warm
    for k in range(1, frames.shape[0]):
        ctx.snapshot()
        t_reb = time_step(ctx, dev[k], eps, cert.CERT_REBUILD, torch)
        ctx.restore()
        t_inc = time_step(ctx, dev[k], eps, cert.CERT_INCREMENTAL, torch)
        f = ctx.features()[0].copy()
        f[7] = prev_ratio
        if k > 1:   # the first step pays one-off costs
            X.append(f)
            T.append([math.log(t_inc), math.log(t_reb)])
        prev_ratio = math.log(t_inc) - math.log(t_reb)
    ctx.close()
    return np.array(X, np.float32), np.array(T, np.float32)


def collect(seeds=16, c1_seeds=100, c3=True, log=print):
    """Transitions of the three plain-method workloads: N=1000 d=2 (20 steps,
    eps 1e-3); N=16000 d=3, five families x eps {1e-4, 1e-3, 5e-3}, 200 steps;
    N=262144 d=3 uniform + clusters, eps 1e-4, 100 steps."""
    import torch
    Xs, Ts, src = [], [], []
    t0 = time.time()
    for seed in range(c1_seeds):
        m = scenes.Motion("uniform_brownian", 1000, 2, 1e-3, seed=10_000 + seed, steps=20)
        X, T = collect_trajectory(m.frames(21), 1e-3, torch=torch)
        Xs.append(X)
        Ts.append(T)
        src += ["c1"] * len(X)
    log(f"c1 done {time.time() - t0:.0f}s rows={sum(len(x) for x in Xs)}")
    for seed in range(seeds):
        for fam in scenes.FAMILIES:
            for eps in (1e-4, 1e-3, 5e-3):
                m = scenes.Motion(fam, 16000, 3, eps, seed=20_000 + seed, steps=200)
                X, T = collect_trajectory(m.frames(201), eps, torch=torch)
                Xs.append(X)
                Ts.append(T)
                src += [f"c2/{fam}/{eps:g}"] * len(X)
        log(f"c2 seed {seed} done {time.time() - t0:.0f}s rows={sum(len(x) for x in Xs)}")
    if c3:
        m = scenes.Motion("uniform_clusters", 262144, 3, 1e-4, seed=30_000, steps=100)
        X, T = collect_trajectory(m.frames(101), 1e-4, torch=torch)
        Xs.append(X)
        Ts.append(T)
        src += ["c3"] * len(X)
    return np.concatenate(Xs), np.concatenate(Ts), np.array(src)


# ----------------------------------------------------------------------------- training

class Trainer:
    """Minibatch Adam on the device through cert_mlp_grad / cert_mlp_adam."""

    def __init__(self, X, T, seed=0, batch=1024):
        import torch
        from . import cert
        self.torch, self.cert = torch, cert
        self.norm_np = normalisation(X)
        self.X = torch.from_numpy(np.ascontiguousarray(X, np.float32)).cuda()
        self.T = torch.from_numpy(np.ascontiguousarray(T, np.float32)).cuda()
        self.norm = torch.from_numpy(self.norm_np).cuda()
        self.params = torch.from_numpy(he_init(seed)).cuda()
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.grad = torch.zeros_like(self.params)
        self.loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        self.batch = int(batch)
        self.work = torch.empty(cert.cert_mlp_workspace_bytes(self.batch) // 4 + 1, dtype=torch.float32,
                                device="cuda")
        self.t = 0

    def fit(self, epochs=60, lr=1e-3):
        n = self.X.shape[0]
        hist = []
        for ep in range(epochs):
            tot, cnt = 0.0, 0
            for a in range(0, n, self.batch):
                b = min(n, a + self.batch)
                self.cert.cert_mlp_grad(self.params, self.norm, self.X[a:b], self.T[a:b], self.grad, self.loss,
                                        self.work)
                self.t += 1
                self.cert.cert_mlp_adam(self.params, self.grad, self.m, self.v, self.t, lr)
                tot += float(self.loss.item()) * (b - a)
                cnt += b - a
            hist.append(tot / cnt)
        return hist

    def params_np(self):
        return self.params.cpu().numpy()


def predict(params, norm, X):
    """Selector outputs (ln t_inc, ln t_reb) for rows X, through cert_mlp_forward."""
    import torch
    from . import cert
    p = torch.from_numpy(np.ascontiguousarray(params, np.float32)).cuda()
    nm = torch.from_numpy(np.ascontiguousarray(norm, np.float32)).cuda()
    Xd = torch.from_numpy(np.ascontiguousarray(X, np.float32)).cuda()
    Y = torch.empty((X.shape[0], 2), dtype=torch.float32, device="cuda")
    cert.cert_mlp_forward(p, nm, Xd, Y)
    return Y.cpu().numpy()


def regret(T_ln, choose_inc):
    """sum_t (T_chosen - min_s T_s) / sum_t min_s T_s on measured times."""
    t = np.exp(T_ln.astype(np.float64))
    chosen = np.where(choose_inc, t[:, 0], t[:, 1])
    best = t.min(axis=1)
    return float((chosen - best).sum() / best.sum())


def decision_margin(Y, T):
    """The margin delta of the rule 'incremental when pred_inc - pred_reb <= delta'
    with the least regret on the given rows (measured times T).  With the rows
    sorted by their predicted difference, choosing incremental on the first k
    rows costs the prefix sum of t_inc plus the suffix sum of t_reb; every k is
    tried and the cheapest taken (ties to the larger k: more incremental
    steps).  The margin is folded into the rebuild head's bias, so the
    device's argmin applies it unchanged."""
    diff = (Y[:, 0] - Y[:, 1]).astype(np.float64)
    t = np.exp(T.astype(np.float64))
    order = np.argsort(diff, kind="stable")
    d, ti, tr = diff[order], t[order, 0], t[order, 1]
    cost = np.concatenate([[0.0], np.cumsum(ti)]) + np.concatenate([np.cumsum(tr[::-1])[::-1], [0.0]])
    k = int(len(cost) - 1 - np.argmin(cost[::-1]))          # last minimum: the most incremental rows
    if k == 0:
        return float(d[0] - 1.0)
    if k == len(d):
        return float(d[-1] + 1.0)
    return float(0.5 * (d[k - 1] + d[k]))


def load(path=WEIGHTS):
    d = np.load(path)
    return d["params"].astype(np.float32), d["norm"].astype(np.float32)


def main():
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    c = sub.add_parser("collect")
    c.add_argument("--out", required=True)
    c.add_argument("--seeds", type=int, default=16)
    c.add_argument("--c1-seeds", type=int, default=100)
    t = sub.add_parser("train")
    t.add_argument("--data", required=True)
    t.add_argument("--out", default=WEIGHTS)
    t.add_argument("--epochs", type=int, default=60)
    t.add_argument("--seed", type=int, default=0)
    args = ap.parse_args()
    if args.cmd == "collect":
        X, T, src = collect(seeds=args.seeds, c1_seeds=args.c1_seeds)
        np.savez_compressed(args.out, X=X, T=T, src=src)
        print(f"{len(X)} transitions -> {args.out}")
        return
    d = np.load(args.data)
    X, T, src = d["X"], d["T"], d["src"]
    rng = np.random.default_rng(args.seed)
    perm = rng.permutation(len(X))
    nval = max(1, len(X) // 10)
    val, tr = perm[:nval], perm[nval:]
    trn = Trainer(X[tr], T[tr], seed=args.seed)
    hist = trn.fit(epochs=args.epochs)
    params, norm = trn.params_np(), trn.norm_np
    delta = decision_margin(predict(params, norm, X[tr]), T[tr])
    params[-1] += np.float32(delta)     # fold the margin into the rebuild head's bias
    Yv = predict(params, norm, X[val])
    vloss = float(np.mean((Yv[:, 0] - T[val, 0]) ** 2 + (Yv[:, 1] - delta - T[val, 1]) ** 2) / 2)
    learned = Yv[:, 0] <= Yv[:, 1]
    meta = {"rows": int(len(X)), "train_rows": int(len(tr)), "val_rows": int(nval), "epochs": args.epochs,
            "decision_margin": float(delta),
            "train_loss_first": hist[0], "train_loss_last": hist[-1], "val_mse": vloss,
            "val_regret_learned": regret(T[val], learned),
            "val_regret_always_incremental": regret(T[val], np.ones(nval, bool)),
            "val_regret_always_rebuild": regret(T[val], np.zeros(nval, bool)),
            "val_regret_threshold": regret(T[val], X[val, 0] < 1.0 / X[val, 2]),
            "sources": sorted(set(str(x).split("/")[0] for x in src))}
    np.savez(args.out, params=params, norm=norm, meta=json.dumps(meta))
    print(json.dumps(meta))


if __name__ == "__main__":
    main()
